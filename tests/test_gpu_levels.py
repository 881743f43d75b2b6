"""Backtrack levels: snapshots taken lazily by the next propagation, restores to
levels with and without a propagation in between, many pending levels."""
import numpy as np
import pytest

from oracle import ct_oracle as O
from paper_2507_18413_gb300 import ct as C
from paper_2507_18413_gb300 import inputs as G
from gpu_helpers import GpuTable, check_index_invariant, compare_call

pytestmark = pytest.mark.gpu


def _table(t=30_000, seed=3):
    dom_lo, dom_size, tup = G.large_table(seed, t, arity=5, d=16)
    return dom_lo, dom_size, O.retained_tuples(tup, dom_lo, dom_size), GpuTable(dom_lo, dom_size, tup)


def _state(gt):
    w, _ = gt.currtable()
    return w.copy(), sorted(gt.index().tolist())


def test_restore_pending_and_materialised_levels():
    dom_lo, dom_size, tup, gt = _table()
    rng = G.Rng(1)
    full = [np.ones(d, bool) for d in dom_size]
    st, root = compare_call(gt, tup, full)
    s_root = _state(gt)
    l0 = gt.save()                       # pending
    l1 = gt.save()                       # pending
    st, a = compare_call(gt, tup, G.reset_step(rng, root)[0])   # snapshots l0 and l1
    assert st == O.OK
    s_a = _state(gt)
    l2 = gt.save()
    l3 = gt.save()                       # pending, nothing propagated since
    gt.restore(l3)                       # no change
    assert _state(gt)[0].tolist() == s_a[0].tolist()
    st, b = compare_call(gt, tup, G.reset_step(rng, a)[0])      # snapshots l2
    assert st == O.OK
    gt.restore(l2)
    assert _state(gt)[0].tolist() == s_a[0].tolist()
    assert _state(gt)[1] == s_a[1]
    # the restored level accepts the domains it was saved with
    st, a2 = compare_call(gt, tup, a)
    assert st == O.OK
    gt.restore(l1)
    assert _state(gt)[0].tolist() == s_root[0].tolist()
    assert _state(gt)[1] == s_root[1]
    st, _ = compare_call(gt, tup, G.delta_step(rng, root)[0])
    gt.restore(l0)
    assert _state(gt)[0].tolist() == s_root[0].tolist()
    gt.close()


def test_many_pending_levels_then_random_restores():
    dom_lo, dom_size, tup, gt = _table(seed=5)
    rng = G.Rng(2)
    full = [np.ones(d, bool) for d in dom_size]
    st, masks = compare_call(gt, tup, full)
    states = []
    for k in range(40):                  # more pending levels than lanes in a warp
        states.append((gt.save(), _state(gt), [m.copy() for m in masks]))
    for k in range(6):
        states.append((gt.save(), _state(gt), [m.copy() for m in masks]))
        new, _ = G.delta_step(rng, masks)
        st, out = compare_call(gt, tup, new)
        if st != O.OK:
            break
        masks = out
    for target in [44, 43, 41, 39, 20, 7, 0]:
        if target >= len(states):
            continue
        lv, s0, m0 = states[target]
        gt.restore(lv)
        s = _state(gt)
        assert s[0].tolist() == s0[0].tolist() and s[1] == s0[1], target
        states = states[:target]
        st, masks = compare_call(gt, tup, m0)
        assert st == O.OK
        states.append((gt.save(), _state(gt), [m.copy() for m in masks]))
    gt.close()


def test_error_state_leaves_the_table_usable():
    dom_lo, dom_size, tup, gt = _table(seed=8)
    rng = G.Rng(4)
    full = [np.ones(d, bool) for d in dom_size]
    st, root = compare_call(gt, tup, full)
    lv = gt.save()
    st, a = compare_call(gt, tup, G.reset_step(rng, root)[0])
    before = _state(gt)
    st, _, _ = gt.propagate(full)        # grows a domain
    assert st == C.CT_ERR_STATE
    assert _state(gt)[0].tolist() == before[0].tolist()
    st, _ = compare_call(gt, tup, G.delta_step(rng, a)[0])
    gt.restore(lv)
    gt.close()


def test_model_search_restores_initial_state():
    csp = O.Csp([0] * 6, [5] * 6)
    rng = G.Rng(9)
    raw = []
    for k in range(4):
        sc = G.random_scope(rng, 6, 3)
        tup = G.distinct_uniform_tuples(G.derive_seed(9, k), [0] * 3, [5] * 3, 40)
        csp.add_table(sc, tup)
        raw.append((sc, tup))
    C.load()
    st, m = C.ct_model_create(csp.dom_lo, csp.dom_size)
    for sc, tup in raw:
        assert C.ct_model_add_table(m, sc, tup) >= 0
    off, _ = C.dom_layout(csp.dom_size)
    st, before = C.ct_model_get_domains(m, int(off[-1]))
    st, d1 = C.ct_search_dfs(m, 6, 0, True)
    st, after = C.ct_model_get_domains(m, int(off[-1]))
    assert before.tolist() == after.tolist()
    st, d2 = C.ct_search_dfs(m, 6, 0, True)
    assert (d1["nodes"], d1["fails"], d1["solutions"]) == (d2["nodes"], d2["fails"], d2["solutions"])
    want = O.dfs(csp)
    assert (d1["nodes"], d1["fails"], d1["solutions"]) == (want.nodes, want.fails, want.solutions)
    C.ct_model_destroy(m)
