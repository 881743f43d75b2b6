"""GPU parity of networks of tables (fixpoint) and of the depth-first search driver.

The GAC closure of a network is unique and the branching rule is deterministic,
so the library and the oracle must agree exactly on domains, nodes, fails,
solutions and the first solution.
"""
import json
import os

import numpy as np
import pytest

from oracle import ct_oracle as O
from paper_2507_18413_gb300 import ct as C
from paper_2507_18413_gb300 import inputs as G
from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu

# both fixpoint paths: the whole fixpoint in one launch, and the host queue
MODES = [pytest.param(0, id="device_fixpoint"), pytest.param(1, id="host_queue")]


class GpuModel:
    def __init__(self, csp: O.Csp, raw_tables, opt=None, host_fixpoint=0):
        if opt is None:
            opt = C.make_options(host_fixpoint=host_fixpoint)
        torch = torch_cuda()
        C.load()
        self.csp = csp
        st, self.h = C.ct_model_create(csp.dom_lo, csp.dom_size, opt=opt, stream=torch.cuda.current_stream())
        assert st == C.CT_OK, C.last_error()
        self.add_status = []
        for scope, tup in raw_tables:
            st = C.ct_model_add_table(self.h, scope, tup)
            assert st >= 0, C.last_error()
            self.add_status.append(st)
        self.off, self.nw = C.dom_layout(csp.dom_size)

    def close(self):
        if self.h:
            C.ct_model_destroy(self.h)
            self.h = None

    def masks(self):
        st, w = C.ct_model_get_domains(self.h, int(self.off[-1]))
        assert st == C.CT_OK
        return C.words_to_masks(w, self.csp.dom_size)

    def set_masks(self, masks):
        return C.ct_model_set_domains(self.h, C.masks_to_words(masks))

    def dfs(self, node_limit=0, count_all=True):
        st, d = C.ct_search_dfs(self.h, self.csp.nvars, node_limit, count_all)
        assert st == C.CT_OK, C.last_error()
        return d


def _build(seed, nvars, ntables, arity, d, t):
    rng = G.Rng(seed)
    csp = O.Csp([0] * nvars, [d] * nvars)
    raw = []
    for k in range(ntables):
        scope = G.random_scope(rng, nvars, arity)
        tt = G.cap_distinct([d] * arity, t)
        tup = G.distinct_uniform_tuples(G.derive_seed(seed, k), [0] * arity, [d] * arity, tt)
        csp.add_table(scope, tup)
        raw.append((scope, tup))
    return csp, raw


def _assert_search_equal(gm, csp, node_limit=0, count_all=True):
    got = gm.dfs(node_limit=node_limit, count_all=count_all)
    want = O.dfs(csp, node_limit=node_limit if node_limit > 0 else 1 << 62, count_all=count_all)
    assert (got["nodes"], got["fails"], got["solutions"]) == (want.nodes, want.fails, want.solutions)
    assert bool(got["complete"]) == want.complete
    assert got["max_depth"] == want.max_depth
    if want.solutions:
        assert got["first_solution"] == want.first_solution
    return got


@pytest.mark.parametrize("mode", MODES)
def test_table1_search(golden_dir, mode):
    with open(os.path.join(golden_dir, "table1.json")) as f:
        g = json.load(f)
    csp = O.Csp(g["scope_dom_lo"], g["scope_dom_size"])
    csp.add_table([0, 1, 2], g["tuples"]["rows"])
    gm = GpuModel(csp, [([0, 1, 2], g["tuples"]["rows"])], host_fixpoint=mode)
    d = _assert_search_equal(gm, csp)
    assert (d["nodes"], d["fails"], d["solutions"]) == (9, 0, 5)
    assert d["first_solution"] == [1, 4, 1]
    gm.close()


@pytest.mark.parametrize("mode", MODES)
def test_triangle_with_failures(mode):
    csp = O.Csp([0, 0, 0], [2, 2, 2])
    raw = [([0, 1], [[0, 0], [1, 1]]), ([1, 2], [[0, 1], [1, 0]]), ([0, 2], [[0, 0], [1, 1]])]
    for s, t in raw:
        csp.add_table(s, t)
    gm = GpuModel(csp, raw, host_fixpoint=mode)
    d = _assert_search_equal(gm, csp)
    assert (d["nodes"], d["fails"], d["solutions"]) == (3, 2, 0)
    gm.close()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("seed", range(8))
def test_random_networks_fixpoint_and_search(seed, mode):
    csp, raw = _build(300 + seed, nvars=7, ntables=5, arity=3, d=5, t=30 + 5 * seed)
    gm = GpuModel(csp, raw, host_fixpoint=mode)
    st = C.ct_model_propagate(gm.h)
    st_o, masks_o, _ = O.gac_network(csp, csp.full_masks())
    assert st == st_o
    if st == C.CT_OK:
        for v, m in enumerate(gm.masks()):
            assert np.array_equal(m, masks_o[v])
    # the search starts from the current (propagated) state and restores it afterwards
    gm.close()
    gm = GpuModel(csp, raw, host_fixpoint=mode)
    _assert_search_equal(gm, csp)
    _assert_search_equal(gm, csp, count_all=False)
    _assert_search_equal(gm, csp, node_limit=7)
    gm.close()


@pytest.mark.parametrize("mode", MODES)
def test_tiny_config_solution_count(mode):
    dom_lo, dom_size, tup = G.tiny_table(seed=1)
    csp = O.Csp(dom_lo, dom_size)
    csp.add_table([0, 1, 2], tup)
    gm = GpuModel(csp, [([0, 1, 2], tup)], host_fixpoint=mode)
    d = gm.dfs()
    assert d["solutions"] == 200 and d["complete"] == 1
    want = O.dfs(csp)
    assert (d["nodes"], d["fails"]) == (want.nodes, want.fails)
    gm.close()


@pytest.mark.parametrize("mode", MODES)
def test_set_domains_save_restore(mode):
    csp, raw = _build(901, nvars=6, ntables=4, arity=3, d=6, t=60)
    gm = GpuModel(csp, raw, host_fixpoint=mode)
    assert C.ct_model_propagate(gm.h) in (C.CT_OK, C.CT_INFEASIBLE)
    st, lv = C.ct_model_save(gm.h)
    assert st == C.CT_OK
    before = gm.masks()
    m = [x.copy() for x in before]
    v = int(np.argmax([x.sum() for x in m]))
    m[v][np.flatnonzero(m[v])[0]] = False
    assert gm.set_masks(m) == C.CT_OK
    st = C.ct_model_propagate(gm.h)
    st_o, mo, _ = O.gac_network(csp, m)
    assert st == st_o
    if st == C.CT_OK:
        for a, b in zip(gm.masks(), mo):
            assert np.array_equal(a, b)
    assert C.ct_model_restore(gm.h, lv) == C.CT_OK
    for a, b in zip(gm.masks(), before):
        assert np.array_equal(a, b)
    # growing domains is refused
    assert gm.set_masks(csp.full_masks()) in (C.CT_OK, C.CT_ERR_STATE)
    gm.close()


@pytest.mark.parametrize("mode", MODES)
def test_large_config_search_prefix(mode):
    """20 variables, d = 32, 8 tables of arity 6 x 1e5 tuples: the first nodes of the tree."""
    csp, raw = _build(2024, nvars=20, ntables=8, arity=6, d=32, t=100_000)
    gm = GpuModel(csp, raw, host_fixpoint=mode)
    _assert_search_equal(gm, csp, node_limit=60)
    gm.close()


def test_autotuned_fixpoint_grid_search():
    """ct_options.autotune picks the fixpoint launch's CTA count with trial
    fixpoints between a save and a restore: the search is unchanged."""
    csp, raw = _build(305, nvars=7, ntables=5, arity=3, d=5, t=55)
    gm = GpuModel(csp, raw, opt=C.make_options(autotune=1))
    _assert_search_equal(gm, csp)
    gm.close()


@pytest.mark.parametrize("seed", range(3))
def test_planning_chain_first_plan(seed):
    """A small planning chain (16 states, 4 actions, 6 steps): the first plan and
    the nodes to reach it equal the oracle's first-fail search."""
    spec = G.planning_csp(seed, states=16, actions=4, horizon=6)
    csp = O.Csp(spec.dom_lo, spec.dom_size)
    raw = []
    for tb in spec.tables:
        csp.add_table(tb.scope, tb.tuples)
        raw.append((tb.scope, tb.tuples))
    gm = GpuModel(csp, raw)
    got = _assert_search_equal(gm, csp, count_all=False)
    assert got["solutions"] == 1
    gm.close()

