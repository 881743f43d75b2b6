"""Helpers for the GPU tests: drive the library through the C ABI and the oracle
side by side on the same seeded inputs."""
import numpy as np

from oracle import ct_oracle as O
from paper_2507_18413_gb300 import ct as C


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("CUDA device not available")
    return torch


class GpuTable:
    """One table on the device plus its domains as a device buffer."""

    def __init__(self, dom_lo, dom_size, tuples, opt=None, stream=None):
        self.torch = torch_cuda()
        C.load()
        self.lo = list(dom_lo)
        self.size = list(dom_size)
        self.arity = len(dom_lo)
        self.tuples = np.asarray(tuples, dtype=np.int32).reshape(-1, self.arity)
        # torch's current stream: the domain copies below and the library's
        # kernels run in stream order
        self.stream = stream if stream is not None else self.torch.cuda.current_stream()
        st, self.h = C.ct_create(self.arity, self.lo, self.size, self.tuples, opt=opt, stream=self.stream)
        assert st >= 0, C.last_error()
        self.create_status = st
        self.off, self.nw = C.dom_layout(self.size)
        self.nch = (self.arity + 31) // 32
        st, self.info = C.ct_get_info(self.h)
        assert st == C.CT_OK
        self.dom = self.torch.zeros(int(self.off[-1]), dtype=self.torch.int32, device="cuda")

    def close(self):
        if self.h:
            C.ct_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_masks(self, masks):
        w = C.masks_to_words(masks).view(np.int32)
        self.dom.copy_(self.torch.from_numpy(w.copy()))

    def get_masks(self):
        w = self.dom.cpu().numpy().view(np.uint32)
        return C.words_to_masks(w, self.size)

    def propagate(self, masks):
        self.set_masks(masks)
        st, ch = C.ct_propagate(self.h, self.dom, self.nch)
        return st, self.get_masks(), ch

    def currtable(self):
        st, w, nz = C.ct_get_currtable(self.h, self.info["words"])
        assert st == C.CT_OK
        return w, nz

    def index(self):
        st, idx = C.ct_get_index(self.h)
        assert st == C.CT_OK
        return idx

    def save(self):
        st, lv = C.ct_save(self.h)
        assert st == C.CT_OK, C.last_error()
        return lv

    def restore(self, lv):
        st = C.ct_restore(self.h, lv)
        assert st == C.CT_OK, C.last_error()

    def stats(self):
        return C.ct_get_call_stats(self.h)[1]


def check_index_invariant(words, idx, nchunks):
    """The index lists each non-zero 128-bit chunk of currTable exactly once."""
    padded = np.zeros(nchunks * 4, dtype=np.uint32)
    padded[: len(words)] = words
    nzc = np.flatnonzero(padded.reshape(-1, 4).any(axis=1))
    assert len(idx) == len(set(idx.tolist())), "duplicate chunk in the index"
    assert sorted(idx.tolist()) == nzc.tolist()


def oracle_step(tup_ret, lo, masks):
    st, out, valid = O.gac_table(tup_ret, lo, masks)
    return st, out, O.currtable_words(valid)


def compare_call(gt, tup_ret, masks, check_table=True):
    """Propagate masks on the GPU and in the oracle; assert identical results.

    Returns (status, new masks)."""
    st_o, out_o, words_o = oracle_step(tup_ret, gt.lo, masks)
    st_g, out_g, ch = gt.propagate(masks)
    assert st_g == st_o, (st_g, st_o, C.last_error())
    if st_o == O.OK:
        for i in range(gt.arity):
            assert np.array_equal(out_g[i], out_o[i]), f"domain of x{i} differs"
        exp_ch = 0
        changed = [not np.array_equal(out_o[i], masks[i]) for i in range(gt.arity)]
        for i, c in enumerate(changed):
            if c:
                assert (int(ch[i >> 5]) >> (i & 31)) & 1, f"x{i} changed but not flagged"
            else:
                assert not (int(ch[i >> 5]) >> (i & 31)) & 1, f"x{i} flagged but unchanged"
            exp_ch += c
        if check_table:
            w, nz = gt.currtable()
            assert np.array_equal(w, words_o), "currTable words differ"
            assert nz == int(np.count_nonzero(words_o))
            check_index_invariant(w, gt.index(), gt.info["chunks"])
        return st_o, out_o
    return st_o, None
