"""GPU parity of short tables (tuples with CT_STAR wildcards) against the
short-table oracle: domains, status and currTable words on every call of
delta/reset streams with backtracking, and searches of networks of short
tables against the oracle's search of the ground tables they stand for."""
import numpy as np
import pytest

from oracle import ct_oracle as O
from oracle import short as S
from paper_2507_18413_gb300 import ct as C
from paper_2507_18413_gb300 import inputs as G
from gpu_helpers import GpuTable, torch_cuda

pytestmark = pytest.mark.gpu


def _call(gt, ret, masks):
    st_o, out_o, valid = S.gac_table_short(ret, gt.lo, masks)
    st_g, out_g, _ = gt.propagate(masks)
    assert st_g == st_o, (st_g, st_o, C.last_error())
    if st_o == O.OK:
        for i in range(gt.arity):
            assert np.array_equal(out_g[i], out_o[i]), f"domain of x{i} differs"
        w, nz = gt.currtable()
        assert np.array_equal(w, O.currtable_words(valid)), "currTable words differ"
        return st_o, out_o
    return st_o, None


@pytest.mark.parametrize("t,arity,d,p", [(300, 3, 6, 0.3), (20_000, 5, 12, 0.15), (150_000, 4, 24, 0.1)])
def test_short_table_streams(t, arity, d, p):
    torch_cuda()
    seed = 4000 + t
    dom_lo, dom_size = [0] * arity, [d] * arity
    tup = G.short_tuples(seed, dom_lo, dom_size, G.cap_distinct(dom_size, t), star_prob=p)
    ret = S.retained_short(tup, dom_lo, dom_size)
    gt = GpuTable(dom_lo, dom_size, tup)
    assert gt.info["short_tuples"] == int((ret == S.STAR).any(axis=1).sum()) > 0
    root = [np.ones(x, bool) for x in dom_size]
    st, out = _call(gt, ret, root)
    assert st == O.OK
    root = out
    gt.save()
    rng = G.Rng(seed)
    masks, depth, seen_delta, seen_reset = root, 0, 0, 0
    for k in range(80):
        gt.save()
        new, i = (G.delta_step if rng.int(2) == 0 else G.reset_step)(rng, masks)
        if i is None:
            new, _ = G.remove_random_values(rng, masks, 1)
        st, out = _call(gt, ret, new)
        s = gt.stats()
        seen_delta += s["delta_vars"]
        seen_reset += s["reset_vars"]
        depth += 1
        if st == O.INFEASIBLE or depth >= 6:
            gt.restore(0)
            gt.save()
            masks, depth = root, 0
        else:
            masks = out
    assert seen_delta > 0 and seen_reset > 0
    gt.close()


def test_all_wildcard_table_supports_everything():
    torch_cuda()
    tup = np.array([[C.CT_STAR, C.CT_STAR], [1, C.CT_STAR]], np.int32)
    gt = GpuTable([0, 0], [3, 4], tup)
    st, out, _ = gt.propagate([np.array([1, 0, 1], bool), np.array([0, 1, 1, 0], bool)])
    assert st == C.CT_OK
    assert out[0].tolist() == [True, False, True] and out[1].tolist() == [False, True, True, False]
    w, _ = gt.currtable()
    assert w.tolist() == [1]  # (1, *) lost its value 1; (*, *) stays
    gt.close()


@pytest.mark.parametrize("seed", range(4))
def test_network_of_short_tables_search(seed):
    torch = torch_cuda()
    rng = G.Rng(7000 + seed)
    nv, d = 6, 4
    sizes = [d] * nv
    ground = O.Csp([0] * nv, sizes)
    st, h = C.ct_model_create([0] * nv, sizes, stream=torch.cuda.current_stream())
    assert st == C.CT_OK
    for k in range(4):
        sc = G.random_scope(rng, nv, 3)
        tup = G.short_tuples(G.derive_seed(7000 + seed, k), [0] * 3, [d] * 3, 12, star_prob=0.2)
        ret = S.retained_short(tup, [0] * 3, [d] * 3)
        ground.add_table(sc, S.expand(ret, [0] * 3, [d] * 3))
        assert C.ct_model_add_table(h, sc, tup) >= 0, C.last_error()
    want = O.dfs(ground)
    st, got = C.ct_search_dfs(h, nv, 0, True)
    assert st == C.CT_OK, C.last_error()
    assert (got["nodes"], got["fails"], got["solutions"]) == (want.nodes, want.fails, want.solutions)
    if want.solutions:
        assert got["first_solution"] == want.first_solution
    st, b, _ = C.ct_search_batch(h, nv, 8, 2, 0, True)
    assert st == C.CT_OK and (b["nodes"], b["solutions"]) == (want.nodes, want.solutions)
    C.ct_model_destroy(h)
