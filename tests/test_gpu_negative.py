"""GPU parity of negative tables (forbidden tuples) against the negative-table
oracle: domains, status and currTable words on every call of streams with
backtracking, and searches of networks with negative tables against the
oracle's search of the allowed tuples."""
import numpy as np
import pytest

from oracle import ct_oracle as O
from oracle import negative as N
from paper_2507_18413_gb300 import ct as C
from paper_2507_18413_gb300 import inputs as G
from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


class NegTable:
    def __init__(self, lo, size, tup):
        self.torch = torch_cuda()
        C.load()
        self.lo, self.size, self.arity = list(lo), list(size), len(lo)
        st, self.h = C.ct_create(self.arity, self.lo, self.size, tup, negative=True,
                                 stream=self.torch.cuda.current_stream())
        assert st == C.CT_OK, C.last_error()
        self.off, _ = C.dom_layout(self.size)
        self.dom = self.torch.zeros(int(self.off[-1]), dtype=self.torch.int32, device="cuda")
        self.info = C.ct_get_info(self.h)[1]

    def propagate(self, masks):
        self.dom.copy_(self.torch.from_numpy(C.masks_to_words(masks).view(np.int32).copy()))
        st, _ = C.ct_propagate(self.h, self.dom, 1)
        return st, C.words_to_masks(self.dom.cpu().numpy().view(np.uint32), self.size)


def _call(nt, ret, masks):
    st_o, out_o, valid = N.gac_table_negative(ret, nt.lo, masks)
    st_g, out_g = nt.propagate(masks)
    assert st_g == st_o, (st_g, st_o, C.last_error())
    if st_o == O.OK:
        for i in range(nt.arity):
            assert np.array_equal(out_g[i], out_o[i]), f"domain of x{i} differs"
        st, w, nz = C.ct_get_currtable(nt.h, nt.info["words"])
        assert np.array_equal(w, O.currtable_words(valid)), "currTable words differ"
        return st_o, out_o
    return st_o, None


@pytest.mark.parametrize("arity,d,t", [(3, 6, 160), (4, 10, 9_500), (3, 40, 63_000)])
def test_negative_table_streams(arity, d, t):
    seed = 5000 + t
    lo, size = [0] * arity, [d] * arity
    tup = G.distinct_uniform_tuples(seed, lo, size, t)
    tup = np.concatenate([tup, tup[:7]])  # duplicates count once
    ret = N.retained_negative(tup, lo, size)
    nt = NegTable(lo, size, tup)
    assert nt.info["tuples"] == len(ret)
    root = [np.ones(x, bool) for x in size]
    st, out = _call(nt, ret, root)
    assert st == O.OK
    root = out
    C.check(C.ct_save(nt.h)[0])
    rng = G.Rng(seed)
    masks, depth, pruned_calls = root, 0, 0
    for k in range(80):
        C.check(C.ct_save(nt.h)[0])
        new, i = (G.delta_step if rng.int(2) == 0 else G.reset_step)(rng, masks)
        if i is None:
            new, _ = G.remove_random_values(rng, masks, 1)
        st, out = _call(nt, ret, new)
        if st == O.OK and any((a != b).any() for a, b in zip(out, new)):
            pruned_calls += 1
        depth += 1
        if st == O.INFEASIBLE or depth >= 6:
            C.check(C.ct_restore(nt.h, 0))
            C.check(C.ct_save(nt.h)[0])
            masks, depth = root, 0
        else:
            masks = out
    assert pruned_calls > 0
    C.ct_destroy(nt.h)


@pytest.mark.parametrize("seed", range(4))
def test_network_with_negative_tables_search(seed):
    torch = torch_cuda()
    rng = G.Rng(8000 + seed)
    nv, d = 6, 3
    sizes = [d] * nv
    allowed = O.Csp([0] * nv, sizes)
    st, h = C.ct_model_create([0] * nv, sizes, stream=torch.cuda.current_stream())
    assert st == C.CT_OK
    for k in range(5):
        sc = G.random_scope(rng, nv, 3)
        forb = G.distinct_uniform_tuples(G.derive_seed(8000 + seed, k), [0] * 3, [d] * 3, 14)
        neg = k % 2 == 0
        if neg:
            ret = N.retained_negative(forb, [0] * 3, [d] * 3)
            allowed.add_table(sc, N.complement(ret, [0] * 3, [d] * 3))
        else:
            allowed.add_table(sc, forb)
        assert C.ct_model_add_table(h, sc, forb, negative=neg) >= 0, C.last_error()
    want = O.dfs(allowed)
    st, got = C.ct_search_dfs(h, nv, 0, True)
    assert st == C.CT_OK, C.last_error()
    assert (got["nodes"], got["fails"], got["solutions"]) == (want.nodes, want.fails, want.solutions)
    if want.solutions:
        assert got["first_solution"] == want.first_solution
    # the batched searches: host-stepped and on the device
    for slots, split in ((4, 1), (16, 3)):
        st, got, _ = C.ct_search_batch(h, nv, slots, split, 0, True)
        assert st == C.CT_OK, C.last_error()
        assert (got["nodes"], got["fails"], got["solutions"]) == (want.nodes, want.fails, want.solutions)
        assert got["max_depth"] == want.max_depth
        if want.solutions:
            assert got["first_solution"] == want.first_solution
        st, got, _ = C.ct_search_batch_device(h, nv, slots, split)
        assert st == C.CT_OK, C.last_error()
        assert (got["nodes"], got["fails"], got["solutions"]) == (want.nodes, want.fails, want.solutions)
    C.ct_model_destroy(h)


def _mixed_network(seed, nv, d, ntables, arity, t_pos, t_neg, every=2):
    """Tables over random scopes, every `every`-th one negative: the library's
    form (forbidden tuples for the negative ones) and the oracle's network of
    allowed tuples (a negative table's complement)."""
    rng = G.Rng(seed)
    allowed = O.Csp([0] * nv, [d] * nv)
    raw = []
    for k in range(ntables):
        sc = G.random_scope(rng, nv, arity)
        neg = k % every == 0
        tt = G.cap_distinct([d] * arity, t_neg if neg else t_pos)
        tup = G.distinct_uniform_tuples(G.derive_seed(seed, k), [0] * arity, [d] * arity, tt)
        if neg:
            ret = N.retained_negative(tup, [0] * arity, [d] * arity)
            allowed.add_table(sc, N.complement(ret, [0] * arity, [d] * arity))
        else:
            allowed.add_table(sc, tup)
        raw.append((sc, tup, neg))
    return allowed, raw


def _mixed_model(allowed, raw, host_fixpoint):
    torch = torch_cuda()
    st, h = C.ct_model_create(allowed.dom_lo, allowed.dom_size, opt=C.make_options(host_fixpoint=host_fixpoint),
                              stream=torch.cuda.current_stream())
    assert st == C.CT_OK, C.last_error()
    for sc, tup, neg in raw:
        assert C.ct_model_add_table(h, sc, tup, negative=neg) >= 0, C.last_error()
    return h


def _model_masks(h, csp):
    off, _ = C.dom_layout(csp.dom_size)
    st, w = C.ct_model_get_domains(h, int(off[-1]))
    assert st == C.CT_OK
    return C.words_to_masks(w, csp.dom_size)


@pytest.mark.parametrize("mode", [pytest.param(0, id="device_fixpoint"), pytest.param(1, id="host_queue")])
@pytest.mark.parametrize("seed", range(4))
def test_network_fixpoint_with_negative_tables(seed, mode):
    """The fixpoint of a network of positive and negative tables equals the
    oracle's GAC closure of the allowed tuples, from the initial domains and
    after random domain cuts (each undone by a restore)."""
    allowed, raw = _mixed_network(8200 + seed, nv=10, d=5, ntables=9, arity=3, t_pos=80, t_neg=45)
    h = _mixed_model(allowed, raw, mode)
    st = C.ct_model_propagate(h)
    st_o, masks_o, _ = O.gac_network(allowed, allowed.full_masks())
    assert st == st_o, C.last_error()
    if st != C.CT_OK:
        C.ct_model_destroy(h)
        return
    for a, b in zip(_model_masks(h, allowed), masks_o):
        assert np.array_equal(a, b)
    rng = np.random.default_rng(seed)
    checked = 0
    for step in range(6):
        st, lv = C.ct_model_save(h)
        assert st == C.CT_OK
        before = _model_masks(h, allowed)
        cut = [m.copy() for m in before]
        for v in rng.choice(allowed.nvars, size=2, replace=False):
            vals = np.flatnonzero(cut[v])
            if len(vals) > 1:
                cut[v][rng.choice(vals, size=len(vals) // 2, replace=False)] = False
        assert C.ct_model_set_domains(h, C.masks_to_words(cut)) == C.CT_OK
        st = C.ct_model_propagate(h)
        st_o, mo, _ = O.gac_network(allowed, cut)
        assert st == st_o, (step, C.last_error())
        if st == C.CT_OK:
            checked += 1
            for a, b in zip(_model_masks(h, allowed), mo):
                assert np.array_equal(a, b), step
        assert C.ct_model_restore(h, lv) == C.CT_OK
        for a, b in zip(_model_masks(h, allowed), before):
            assert np.array_equal(a, b)
    C.ct_model_destroy(h)


@pytest.mark.parametrize("seed", range(3))
def test_negative_only_network_reaches_the_closure(seed):
    """Networks of negative tables only (each pass of one may enable another
    removal by the same table): the one-launch fixpoint, the host queue and
    the oracle agree, and so do the searches."""
    allowed, raw = _mixed_network(8300 + seed, nv=7, d=4, ntables=6, arity=3, t_pos=0, t_neg=30, every=1)
    st_o, masks_o, _ = O.gac_network(allowed, allowed.full_masks())
    want = O.dfs(allowed)
    for mode in (0, 1):
        h = _mixed_model(allowed, raw, mode)
        st = C.ct_model_propagate(h)
        assert st == st_o, C.last_error()
        if st == C.CT_OK:
            for a, b in zip(_model_masks(h, allowed), masks_o):
                assert np.array_equal(a, b)
        C.ct_model_destroy(h)
        h = _mixed_model(allowed, raw, mode)
        st, got = C.ct_search_dfs(h, allowed.nvars, 0, True)
        assert st == C.CT_OK, C.last_error()
        assert (got["nodes"], got["fails"], got["solutions"]) == (want.nodes, want.fails, want.solutions)
        C.ct_model_destroy(h)


def test_negative_table_arguments():
    torch_cuda()
    C.load()
    st, _ = C.ct_create(2, [0, 0], [3, 3], np.zeros((0, 2), np.int32), negative=True)
    assert st == C.CT_ERR_ARG
    st, _ = C.ct_create(2, [0, 0], [3, 3], np.array([[C.CT_STAR, 1]], np.int32), negative=True)
    assert st == C.CT_ERR_ARG
    st, h = C.ct_create(2, [0, 0], [3, 3], np.array([[5, 5], [1, 1]], np.int32), negative=True)
    assert st == C.CT_OK and C.ct_get_info(h)[1]["tuples"] == 1
    C.ct_destroy(h)
