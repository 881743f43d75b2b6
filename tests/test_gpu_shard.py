"""GPU parity of one table split into word-range shards (the data-parallel
split of a single table, run on one device) against the oracle's GAC of the
whole table: status, domains, changed variables and the concatenated
currTable words on every call of delta/reset streams with backtracking, for
several shard counts, ragged last shards and shards that run empty."""
import numpy as np
import pytest

from oracle import ct_oracle as O
from paper_2507_18413_gb300 import ct as C
from paper_2507_18413_gb300 import inputs as G
from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


class Sharded:
    def __init__(self, lo, size, tup, K, opt=None):
        self.torch = torch_cuda()
        C.load()
        self.lo, self.size, self.arity = list(lo), list(size), len(lo)
        st, self.h = C.ct_sharded_create(self.arity, self.lo, self.size, tup, K, opt=opt,
                                         stream=self.torch.cuda.current_stream())
        assert st == C.CT_OK, C.last_error()
        self.off, _ = C.dom_layout(self.size)
        self.dom = self.torch.zeros(int(self.off[-1]), dtype=self.torch.int32, device="cuda")
        self.nch = (self.arity + 31) // 32

    def propagate(self, masks):
        self.dom.copy_(self.torch.from_numpy(C.masks_to_words(masks).view(np.int32).copy()))
        st, ch = C.ct_sharded_propagate(self.h, self.dom, self.nch)
        return st, ch, C.words_to_masks(self.dom.cpu().numpy().view(np.uint32), self.size)

    def close(self):
        C.ct_sharded_destroy(self.h)


def _call(sh, ret, masks):
    st_o, out_o, valid = O.gac_table(ret, sh.lo, masks)
    st_g, ch, out_g = sh.propagate(masks)
    assert st_g == st_o, (st_g, st_o, C.last_error())
    if st_o != O.OK:
        return st_o, None
    for i in range(sh.arity):
        assert np.array_equal(out_g[i], out_o[i]), f"domain of x{i} differs"
        changed = bool((ch[i // 32] >> (i % 32)) & 1)
        assert changed == (not np.array_equal(out_o[i], masks[i])), f"changed bit of x{i}"
    st, w, nz = C.ct_sharded_get_currtable(sh.h, (len(ret) + 31) // 32)
    want = O.currtable_words(valid)
    assert np.array_equal(w, want), "concatenated currTable words differ"
    assert nz == int(np.count_nonzero(want))
    return st_o, out_o


@pytest.mark.parametrize("arity,d,t,K", [(3, 8, 200, 2), (4, 12, 5_000, 3), (6, 32, 100_000, 7),
                                         (5, 16, 40_000, 16)])
def test_sharded_streams_match_the_whole_table(arity, d, t, K):
    seed = 6100 + t + K
    lo, size = [0] * arity, [d] * arity
    tup = G.distinct_uniform_tuples(seed, lo, size, G.cap_distinct(size, t))
    ret = O.retained_tuples(tup, lo, size)
    sh = Sharded(lo, size, tup, K)
    root = [np.ones(x, bool) for x in size]
    st, out = _call(sh, ret, root)
    assert st == O.OK
    root = out
    C.check(C.ct_sharded_save(sh.h)[0])
    rng = G.Rng(seed)
    masks, depth, fails = root, 0, 0
    for k in range(60):
        C.check(C.ct_sharded_save(sh.h)[0])
        new, i = (G.delta_step if rng.int(2) == 0 else G.reset_step)(rng, masks)
        if i is None:
            new, _ = G.remove_random_values(rng, masks, 1)
        st, out = _call(sh, ret, new)
        depth += 1
        if st == O.INFEASIBLE or depth >= 6:
            fails += st == O.INFEASIBLE
            C.check(C.ct_sharded_restore(sh.h, 0))
            C.check(C.ct_sharded_save(sh.h)[0])
            masks, depth = root, 0
        else:
            masks = out
    sh.close()


def test_shards_that_run_empty():
    """Tuples ordered by their first value: fixing x0 empties every shard but
    the ones holding that value's tuples; the others support nothing and the
    combined domains are still the GAC of the whole table."""
    torch_cuda()
    lo, size = [0, 0, 0], [4, 16, 16]
    tup = G.distinct_uniform_tuples(6301, lo, size, 800)
    tup = tup[np.argsort(tup[:, 0], kind="stable")]
    ret = O.retained_tuples(tup, lo, size)
    sh = Sharded(lo, size, tup, 5)
    st, root = _call(sh, ret, [np.ones(x, bool) for x in size])
    assert st == O.OK
    C.check(C.ct_sharded_save(sh.h)[0])
    for v in np.flatnonzero(root[0]):
        masks = [m.copy() for m in root]
        masks[0][:] = False
        masks[0][v] = True
        st, out = _call(sh, ret, masks)
        empty = 0
        for k in range(5):
            s, tab = C.ct_sharded_get_shard(sh.h, k)
            assert s == C.CT_OK
            empty += C.ct_get_info(tab)[1]["live_chunks"] == 0
        assert empty >= 1, "some shard should hold none of the value's tuples"
        C.check(C.ct_sharded_restore(sh.h, 0))
        C.check(C.ct_sharded_save(sh.h)[0])
    # a domain emptied by every shard: the whole table fails
    masks = [m.copy() for m in root]
    masks[1][:] = False
    masks[1][np.flatnonzero(root[1])[0]] = True
    st_o, _, _ = O.gac_table(ret, lo, masks)
    st_g, _, _ = sh.propagate(masks)
    assert st_g == st_o
    sh.close()


def test_sharded_arguments():
    torch_cuda()
    C.load()
    st, _ = C.ct_sharded_create(2, [0, 0], [3, 3], np.array([[0, 0], [1, 1]], np.int32), 2)
    assert st == C.CT_ERR_ARG  # two shards of one 128-tuple chunk
    st, _ = C.ct_sharded_create(2, [0, 0], [3, 3], np.array([[5, 5]], np.int32), 1)
    assert st == C.CT_INFEASIBLE
    st, h = C.ct_sharded_create(2, [0, 0], [3, 3], np.array([[0, 1], [2, 2]], np.int32), 1)
    assert st == C.CT_OK
    assert C.ct_sharded_get_shard(h, 1)[0] == C.CT_ERR_ARG
    C.ct_sharded_destroy(h)
