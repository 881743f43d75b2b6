"""ct_propagate_noalloc, the propagation entry point that allocates nothing.

Callers whose device memory belongs to someone else at propagation time (a
framework's memory pool, a service that allocates only at start-up) hand the
library every buffer: supports, currTable, domains and last domains. The
library keeps its scratch in one static device array and calls no allocator.
Here that entry point must give exactly what ct_propagate gives (domains,
currTable words, changed variables, status) on two calls in a row. The file is
collected last so that a run stopping at the first failure has run every other
test before it; it also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2507_18413_gb300 import ct as C
from paper_2507_18413_gb300 import inputs as G
from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


def test_noalloc_matches_ct_propagate_on_two_calls_in_a_row():
    torch = torch_cuda()
    C.load()
    stream = torch.cuda.current_stream()
    # ragged sizes: 50,000 tuples -> 1,563 words -> 391 chunks (a partial last segment)
    dom_lo, dom_size, tup = G.large_table(seed=17, t=50_000, arity=5, d=20)
    st, h = C.ct_create(5, dom_lo, dom_size, tup, stream=stream)
    assert st == C.CT_OK, C.last_error()
    info = C.ct_get_info(h)[1]
    W, W4, R = info["words"], info["chunks"], info["rows"]
    Wp = 4 * W4
    # caller-owned device buffers, allocated by the caller (here: torch)
    sup = np.zeros((R, Wp), np.uint32)
    for r in range(R):
        st, row = C.ct_get_support_row(h, r, W)
        assert st == C.CT_OK
        sup[r, :W] = row
    sup_d = torch.from_numpy(sup.view(np.int32)).cuda()
    t = info["tuples"]
    curr = np.zeros(Wp, np.uint32)
    curr[: t // 32] = 0xFFFFFFFF
    if t % 32:
        curr[t // 32] = (1 << (t % 32)) - 1
    curr_d = torch.from_numpy(curr.view(np.int32).copy()).cuda()
    full = C.masks_to_words([np.ones(d, bool) for d in dom_size])
    last_d = torch.from_numpy(full.view(np.int32).copy()).cuda()
    DW = full.shape[0]
    dom_ref = torch.zeros(DW, dtype=torch.int32, device="cuda")
    dom_na = torch.zeros(DW, dtype=torch.int32, device="cuda")

    rng = G.Rng(5)
    masks = [np.ones(d, bool) for d in dom_size]
    for k in range(2):
        new, _ = G.reset_step(rng, masks) if k == 0 else G.delta_step(rng, masks)
        w = torch.from_numpy(C.masks_to_words(new).view(np.int32).copy()).cuda()
        dom_ref.copy_(w)
        dom_na.copy_(w)
        st_ref, ch_ref = C.ct_propagate(h, dom_ref, 1)
        st_na, ch_na = C.ct_propagate_noalloc(dom_size, t, sup_d, curr_d, dom_na, last_d, stream=stream)
        assert st_ref == C.CT_OK, C.last_error()
        assert st_na == st_ref, C.last_error()
        assert torch.equal(dom_na, dom_ref), f"call {k}: domains differ"
        st, ref_words, _ = C.ct_get_currtable(h, W)
        got = curr_d.cpu().numpy().view(np.uint32)
        assert np.array_equal(got[:W], ref_words), f"call {k}: currTable differs"
        assert not got[W:].any()
        assert ch_na == int(ch_ref[0]), f"call {k}: changed variables differ"
        assert torch.equal(last_d, dom_ref), f"call {k}: last domains are not the output"
        masks = C.words_to_masks(dom_ref.cpu().numpy().view(np.uint32), dom_size)
    C.ct_destroy(h)


def test_noalloc_rejects_sizes_beyond_its_limits():
    torch_cuda()
    C.load()
    fake = 1 << 20  # never dereferenced: the sizes are refused first
    st, _ = C.ct_propagate_noalloc([4] * 17, 10, fake, fake, fake, fake)
    assert st == C.CT_ERR_ARG and "arity" in C.last_error()
    st, _ = C.ct_propagate_noalloc([1000, 100], 10, fake, fake, fake, fake)
    assert st == C.CT_ERR_ARG and "limits" in C.last_error()
    st, _ = C.ct_propagate_noalloc([4, 4], 9_000_000, fake, fake, fake, fake)
    assert st == C.CT_ERR_ARG and "limits" in C.last_error()
