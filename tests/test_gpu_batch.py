"""GPU parity of the batched search (ct_search_batch).

Counting every solution visits the whole tree whatever the order of the
nodes, so with count_all and no node limit the batched search must give the
oracle's depth-first counts exactly: nodes, fails, solutions, maximum depth,
and the first solution in depth-first order. Asked for the first solution
only, it must return the oracle's first solution. Splits at depth 0 (one open
node, the rest by handing over right branches between slots), at depths with
fewer and with more open nodes than slots, and with more tables in a round
than the fixpoint kernel keeps in shared memory.
"""
import numpy as np
import pytest

from oracle import ct_oracle as O
from paper_2507_18413_gb300 import ct as C
from paper_2507_18413_gb300 import inputs as G
from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


def _model(csp, raw, host_fixpoint=0):
    torch = torch_cuda()
    C.load()
    opt = C.make_options(host_fixpoint=host_fixpoint)
    st, h = C.ct_model_create(csp.dom_lo, csp.dom_size, opt=opt, stream=torch.cuda.current_stream())
    assert st == C.CT_OK, C.last_error()
    for scope, tup in raw:
        assert C.ct_model_add_table(h, scope, tup) >= 0, C.last_error()
    return h


def _random(seed, nvars, ntables, arity, d, t):
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


def _domains(h, csp):
    off, _ = C.dom_layout(csp.dom_size)
    st, w = C.ct_model_get_domains(h, int(off[-1]))
    assert st == C.CT_OK
    return w.copy()


def _batch(h, csp, slots, split, node_limit=0, count_all=True):
    st, d, info = C.ct_search_batch(h, csp.nvars, slots, split, node_limit, count_all)
    assert st == C.CT_OK, C.last_error()
    return d, info


def _assert_counts(got, want):
    assert (got["nodes"], got["fails"], got["solutions"]) == (want.nodes, want.fails, want.solutions)
    assert got["max_depth"] == want.max_depth
    assert bool(got["complete"]) == want.complete
    if want.solutions:
        assert got["first_solution"] == want.first_solution


SHAPES = [(1, 0), (4, 0), (4, 2), (16, 3), (7, 5), (64, 1)]


@pytest.mark.parametrize("slots,split", SHAPES)
@pytest.mark.parametrize("seed", range(6))
def test_batch_counts_equal_the_oracle_search(seed, slots, split):
    csp, raw = _random(300 + seed, nvars=7, ntables=5, arity=3, d=5, t=30 + 5 * seed)
    want = O.dfs(csp, count_all=True)
    h = _model(csp, raw)
    before = _domains(h, csp)
    got, info = _batch(h, csp, slots, split)
    _assert_counts(got, want)
    assert info["split_nodes"] + info["slot_nodes"] == got["nodes"]
    assert np.array_equal(_domains(h, csp), before), "the model's domains changed"
    # the model is intact: the plain search still agrees, and a second batched call too
    st, d = C.ct_search_dfs(h, csp.nvars, 0, True)
    assert st == C.CT_OK and (d["nodes"], d["solutions"]) == (want.nodes, want.solutions)
    got2, _ = _batch(h, csp, slots, split)
    _assert_counts(got2, want)
    C.ct_model_destroy(h)


@pytest.mark.parametrize("slots,split", [(3, 1), (8, 0)])
def test_batch_table1(golden_dir, slots, split):
    import json
    import os
    with open(os.path.join(golden_dir, "table1.json")) as f:
        g = json.load(f)
    csp = O.Csp(g["scope_dom_lo"], g["scope_dom_size"])
    csp.add_table([0, 1, 2], g["tuples"]["rows"])
    h = _model(csp, [([0, 1, 2], g["tuples"]["rows"])])
    got, _ = _batch(h, csp, slots, split)
    assert (got["nodes"], got["fails"], got["solutions"]) == (9, 0, 5)
    assert got["first_solution"] == [1, 4, 1]
    C.ct_model_destroy(h)


def test_batch_triangle_all_nodes_fail():
    csp = O.Csp([0, 0, 0], [2, 2, 2])
    raw = [([0, 1], [[0, 0], [1, 1]]), ([1, 2], [[0, 1], [1, 0]]), ([0, 2], [[0, 0], [1, 1]])]
    for s, t in raw:
        csp.add_table(s, t)
    h = _model(csp, raw)
    for slots, split in [(1, 0), (2, 1), (4, 0)]:
        got, _ = _batch(h, csp, slots, split)
        assert (got["nodes"], got["fails"], got["solutions"]) == (3, 2, 0)
    C.ct_model_destroy(h)


def test_batch_tiny_config_counts_200_solutions():
    dom_lo, dom_size, tup = G.tiny_table(seed=1)
    csp = O.Csp(dom_lo, dom_size)
    csp.add_table([0, 1, 2], tup)
    want = O.dfs(csp)
    h = _model(csp, [([0, 1, 2], tup)])
    for slots, split in [(8, 2), (32, 4), (128, 0)]:
        got, info = _batch(h, csp, slots, split)
        _assert_counts(got, want)
        assert got["solutions"] == 200
    C.ct_model_destroy(h)


@pytest.mark.parametrize("seed", range(4))
def test_batch_first_solution_mode(seed):
    csp, raw = _random(500 + seed, nvars=8, ntables=6, arity=3, d=5, t=40)
    want = O.dfs(csp, count_all=False)
    h = _model(csp, raw)
    for slots, split in [(4, 2), (16, 0), (9, 4)]:
        got, _ = _batch(h, csp, slots, split, count_all=False)
        assert got["complete"] == 1
        assert (got["solutions"] > 0) == (want.solutions > 0)
        if want.solutions:
            assert got["first_solution"] == want.first_solution
        else:
            assert (got["nodes"], got["fails"]) == (want.nodes, want.fails)
    C.ct_model_destroy(h)


def test_batch_node_limit():
    csp, raw = _random(303, nvars=7, ntables=5, arity=3, d=5, t=45)
    full = O.dfs(csp)
    assert full.nodes > 1000
    h = _model(csp, raw)
    for slots, split, limit in [(4, 2, 25), (8, 0, 40), (2, 6, 10)]:
        got, _ = _batch(h, csp, slots, split, node_limit=limit)
        assert got["nodes"] == limit and got["complete"] == 0
        assert got["fails"] + got["solutions"] <= limit
    got, _ = _batch(h, csp, 4, 2, node_limit=full.nodes + 5)
    _assert_counts(got, full)
    C.ct_model_destroy(h)


def test_batch_rounds_longer_than_the_shared_prefix():
    """136 slots x 16 tables: the first step propagates 2,176 tables in one round
    (168 open nodes at depth 8), more than the kernel's shared-memory prefix holds."""
    csp, raw = _random(4242, nvars=12, ntables=16, arity=3, d=5, t=60)
    want = O.dfs(csp)
    assert want.complete and want.nodes == 3993
    h = _model(csp, raw)
    got, info = _batch(h, csp, 136, 8)
    _assert_counts(got, want)
    assert info["open_nodes"] == 168
    got, info = _batch(h, csp, 24, 0)
    _assert_counts(got, want)
    assert info["steals"] > 0
    C.ct_model_destroy(h)


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_multi_segment_tables_match_the_plain_search(mode):
    """28 tables of 5,000 tuples (40 chunks: two segments each); both fixpoint modes of the model."""
    csp, raw = _random(91, nvars=8, ntables=28, arity=4, d=10, t=5000)
    h = _model(csp, raw, host_fixpoint=mode)
    st, plain = C.ct_search_dfs(h, csp.nvars, 0, True)
    assert st == C.CT_OK and plain["complete"] == 1
    got, info = _batch(h, csp, 32, 3)
    for k in ("nodes", "fails", "solutions", "max_depth", "complete", "first_solution"):
        assert got[k] == plain[k], k
    C.ct_model_destroy(h)


def test_batch_without_tables_and_bad_arguments():
    csp = O.Csp([0, 0], [2, 3])
    want = O.dfs(csp)
    h = _model(csp, [])
    got, _ = _batch(h, csp, 4, 1)
    _assert_counts(got, want)
    assert C.ct_search_batch(h, csp.nvars, 0, 1)[0] == C.CT_ERR_ARG
    assert C.ct_search_batch(h, csp.nvars, 4, 65)[0] == C.CT_ERR_ARG
    C.ct_model_destroy(h)


@pytest.mark.parametrize("seed", range(4))
def test_batch_any_solution_mode(seed):
    """count_all = 2 stops at the first solution any slot finds: it must be a
    solution of every table; without solutions the whole tree is visited."""
    csp, raw = _random(500 + seed, nvars=8, ntables=6, arity=3, d=5, t=40)
    want = O.dfs(csp)
    h = _model(csp, raw)
    for slots, split in [(4, 2), (16, 0), (9, 4)]:
        got, _ = _batch(h, csp, slots, split, count_all="any")
        assert got["complete"] == 1
        assert (got["solutions"] > 0) == (want.solutions > 0)
        if want.solutions:
            sol = got["first_solution"]
            for scope, tup in csp.tables:
                assert any(all(int(row[k]) == sol[v] for k, v in enumerate(scope)) for row in tup)
        else:
            assert (got["nodes"], got["fails"]) == (want.nodes, want.fails)
    assert C.ct_search_batch(h, csp.nvars, 4, 1, 0, 3)[0] == C.CT_ERR_ARG
    C.ct_model_destroy(h)


# --------------------------------------------------------------------------
# split at a number of assignments (ct_search_batch_assign)
# --------------------------------------------------------------------------

def _open_nodes_by_assignments(csp, depth):
    """Oracle count of the nodes that reach `depth` assignments (left branches)
    in the depth-first tree, i.e. the open nodes of the split."""
    count = 0

    def node(m, a):
        nonlocal count
        if a == depth:
            count += 1
            return
        st, m2, _ = O.gac_network(csp, m)
        if st == O.INFEASIBLE:
            return
        x = O.select_first_fail(m2)
        if x is None:
            return
        v = int(np.flatnonzero(m2[x])[0])
        left = [mm.copy() for mm in m2]
        left[x] = np.zeros_like(m2[x])
        left[x][v] = True
        right = [mm.copy() for mm in m2]
        right[x][v] = False
        node(left, a + 1)
        node(right, a)

    node(csp.full_masks(), 0)
    return count


@pytest.mark.parametrize("slots,depth", [(4, 1), (16, 2), (64, 3), (5, 4)])
@pytest.mark.parametrize("seed", range(4))
def test_batch_assignment_split_counts_equal_the_oracle_search(seed, slots, depth):
    csp, raw = _random(700 + seed, nvars=7, ntables=5, arity=3, d=5, t=35 + 5 * seed)
    want = O.dfs(csp, count_all=True)
    h = _model(csp, raw)
    st, got, info = C.ct_search_batch(h, csp.nvars, slots, depth, 0, True, split_assignments=True)
    assert st == C.CT_OK, C.last_error()
    _assert_counts(got, want)
    assert info["split_nodes"] + info["slot_nodes"] == got["nodes"]
    assert info["open_nodes"] == _open_nodes_by_assignments(csp, depth)
    # first solution mode returns the depth-first first solution
    want1 = O.dfs(csp, count_all=False)
    st, got1, _ = C.ct_search_batch(h, csp.nvars, slots, depth, 0, False, split_assignments=True)
    assert st == C.CT_OK
    if want1.solutions:
        assert got1["first_solution"] == want1.first_solution
    C.ct_model_destroy(h)


def test_batch_assignment_split_bad_arguments():
    csp, raw = _random(710, nvars=5, ntables=3, arity=3, d=4, t=20)
    h = _model(csp, raw)
    for depth, mode in [(0, True), (17, True), (3, "any")]:
        st, _, _ = C.ct_search_batch(h, csp.nvars, 4, depth, 0, mode, split_assignments=True)
        assert st == C.CT_ERR_ARG
    C.ct_model_destroy(h)


# --------------------------------------------------------------------------
# the slots' search run on the device (ct_search_batch_device)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("slots,split", [(1, 0), (4, 2), (16, 3), (7, 5), (64, 1)])
@pytest.mark.parametrize("seed", range(5))
def test_device_search_counts_equal_the_oracle_search(seed, slots, split):
    csp, raw = _random(300 + seed, nvars=7, ntables=5, arity=3, d=5, t=30 + 5 * seed)
    want = O.dfs(csp, count_all=True)
    h = _model(csp, raw)
    before = _domains(h, csp)
    st, got, info = C.ct_search_batch_device(h, csp.nvars, slots, split)
    assert st == C.CT_OK, C.last_error()
    _assert_counts(got, want)
    assert info["split_nodes"] + info["slot_nodes"] == got["nodes"]
    assert np.array_equal(_domains(h, csp), before), "the model's domains changed"
    # the model and the host-stepped search are intact afterwards
    got2, _ = _batch(h, csp, slots, split)
    _assert_counts(got2, want)
    st, got3, _ = C.ct_search_batch_device(h, csp.nvars, slots, split)
    assert st == C.CT_OK
    _assert_counts(got3, want)
    C.ct_model_destroy(h)


def test_device_search_tiny_config_and_unconstrained_variable():
    """The config-1 CSP (200 solutions), and a network with a variable that no
    table holds (its branches propagate nothing)."""
    dom_lo, dom_size, tup = G.tiny_table(seed=1)
    csp = O.Csp(dom_lo, dom_size)
    csp.add_table([0, 1, 2], tup)
    want = O.dfs(csp)
    h = _model(csp, [([0, 1, 2], tup)])
    for slots, split in [(8, 2), (32, 4), (128, 0)]:
        st, got, _ = C.ct_search_batch_device(h, csp.nvars, slots, split)
        assert st == C.CT_OK, C.last_error()
        _assert_counts(got, want)
        assert got["solutions"] == 200
    C.ct_model_destroy(h)
    csp2, raw2 = _random(321, nvars=6, ntables=3, arity=2, d=4, t=10)
    free = O.Csp([0] * 7, [4] * 7)  # variable 6 in no table
    for scope, tup in raw2:
        free.add_table(scope, tup)
    want2 = O.dfs(free)
    h2 = _model(free, raw2)
    st, got, _ = C.ct_search_batch_device(h2, free.nvars, 8, 2)
    assert st == C.CT_OK, C.last_error()
    _assert_counts(got, want2)
    C.ct_model_destroy(h2)


def test_device_search_node_limit_and_bad_arguments():
    csp, raw = _random(303, nvars=7, ntables=5, arity=3, d=5, t=45)
    full = O.dfs(csp)
    h = _model(csp, raw)
    for slots, split, limit in [(4, 2, 25), (8, 0, 40), (2, 6, 10), (16, 3, 500)]:
        st, got, _ = C.ct_search_batch_device(h, csp.nvars, slots, split, limit)
        assert st == C.CT_OK, C.last_error()
        assert got["nodes"] == min(limit, full.nodes)
        assert got["fails"] + got["solutions"] <= got["nodes"]
    st, got, _ = C.ct_search_batch_device(h, csp.nvars, 4, 2, full.nodes + 5)
    _assert_counts(got, full)
    st, _, _ = C.ct_search_batch_device(h, csp.nvars, 0, 2)
    assert st == C.CT_ERR_ARG
    C.ct_model_destroy(h)
