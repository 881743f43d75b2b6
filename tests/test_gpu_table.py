"""GPU parity of single-table propagation against the CPU oracle (through the C ABI).

Bit-exact on: status (OK / INFEASIBLE), filtered domains, changed-variable
mask, currTable words, the non-zero index set, and save/restore round trips.
"""
import json
import os

import numpy as np
import pytest

from oracle import ct_oracle as O
from paper_2507_18413_gb300 import ct as C
from paper_2507_18413_gb300 import inputs as G
from gpu_helpers import GpuTable, check_index_invariant, compare_call, oracle_step, torch_cuda

pytestmark = pytest.mark.gpu


def _golden(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        return json.load(f)


# --------------------------------------------------------------------------
# Table 1 worked example
# --------------------------------------------------------------------------

def test_table1_supports_and_currtable(golden_dir):
    g = _golden(golden_dir, "table1.json")
    lo, sz, tup = g["scope_dom_lo"], g["scope_dom_size"], g["tuples"]["rows"]
    gt = GpuTable(lo, sz, tup)
    assert gt.create_status == C.CT_OK
    sup = O.supports_matrix(tup, lo, sz)
    for r in range(sup.shape[0]):
        st, row = C.ct_get_support_row(gt.h, r, gt.info["words"])
        assert st == C.CT_OK
        assert row.tolist() == O.pack_words(sup[r]).tolist(), r
    # dom(x1) = {1}: currTable 01010, dom(x2) = {2,4}, dom(x3) = {1,3}
    masks = [np.array([True, False, False, False]), np.ones(4, bool), np.ones(4, bool)]
    compare_call(gt, O.retained_tuples(tup, lo, sz), masks)
    w, _ = gt.currtable()
    assert w.tolist() == [0b01010]
    gt.close()


# --------------------------------------------------------------------------
# config 1 stream: arity 3, d = 8, 200 tuples, 1,000 calls
# --------------------------------------------------------------------------

def _tiny_stream(seed, calls, opt=None, check_every=1):
    dom_lo, dom_size, tup = G.tiny_table(seed=seed)
    tup_ret = O.retained_tuples(tup, dom_lo, dom_size)
    gt = GpuTable(dom_lo, dom_size, tup, opt=opt)
    rng = G.Rng(G.derive_seed(seed, 1000))
    root = [np.ones(d, bool) for d in dom_size]
    gt.save()  # level 0 = root
    masks = root
    stack = []
    counts = {"ok": 0, "fail": 0, "restores": 0}
    for k in range(calls):
        lv = gt.save()
        stack.append((lv, masks))
        new, _ = G.remove_random_values(rng, masks, 1 + rng.int(4))
        st, out = compare_call(gt, tup_ret, new, check_table=(k % check_every == 0))
        if st == O.INFEASIBLE or all(m.sum() == 1 for m in out):
            counts["fail" if st == O.INFEASIBLE else "ok"] += 1
            gt.restore(0)
            gt.save()
            stack = []
            masks = root
            counts["restores"] += 1
        else:
            counts["ok"] += 1
            masks = out
    gt.close()
    return counts


def test_tiny_stream_1000_calls():
    counts = _tiny_stream(seed=1, calls=1000)
    assert counts["fail"] > 0 and counts["ok"] > 0 and counts["restores"] > 0


@pytest.mark.parametrize("opt", [dict(grid_blocks=1), dict(grid_blocks=2), dict(no_residues=1),
                                 dict(grid_blocks=3, no_residues=1)])
def test_tiny_stream_options(opt):
    _tiny_stream(seed=2, calls=150, opt=C.make_options(**opt))


# --------------------------------------------------------------------------
# config 2 streams: arity 6, d = 32, delta and reset steps, dives with restore
# --------------------------------------------------------------------------

def _large_stream(t, calls, seed, opt=None, check_every=1, depth=8):
    dom_lo, dom_size, tup = G.large_table(seed, t)
    tup_ret = O.retained_tuples(tup, dom_lo, dom_size)
    gt = GpuTable(dom_lo, dom_size, tup, opt=opt)
    rng = G.Rng(G.derive_seed(seed, 77))
    root = [np.ones(d, bool) for d in dom_size]
    # first call: full domains, filter only
    st, out = compare_call(gt, tup_ret, root)
    assert st == O.OK
    root = out
    gt.save()
    masks = root
    d = 0
    seen = {"delta": 0, "reset": 0, "fail": 0, "early": 0, "calls": 0}
    for k in range(calls):
        gt.save()
        if rng.int(2) == 0:
            new, i = G.delta_step(rng, masks)
        else:
            new, i = G.reset_step(rng, masks)
        if i is None:
            new, _ = G.remove_random_values(rng, masks, 1)
        st, out = compare_call(gt, tup_ret, new, check_table=(k % check_every == 0))
        s = gt.stats()
        seen["delta"] += s["delta_vars"]
        seen["reset"] += s["reset_vars"]
        seen["early"] += s["early_filter"]
        seen["calls"] += 1
        d += 1
        if st == O.INFEASIBLE or d >= depth:
            seen["fail"] += st == O.INFEASIBLE
            gt.restore(0)
            gt.save()
            masks, d = root, 0
        else:
            masks = out
    gt.close()
    return seen


def test_large_stream_1e5():
    seen = _large_stream(100_000, calls=200, seed=11)
    assert seen["delta"] > 0 and seen["reset"] > 0


def test_autotuned_launch_shape_gives_the_same_results():
    """ct_options.autotune times trial propagations at creation (between a save
    and a restore): the table must start from its creation state and match the
    oracle on every call."""
    seen = _large_stream(100_000, calls=100, seed=21, opt=C.make_options(autotune=1))
    assert seen["delta"] > 0 and seen["reset"] > 0
    dom_lo, dom_size, tup = G.large_table(21, 100_000)
    gt = GpuTable(dom_lo, dom_size, tup, opt=C.make_options(autotune=1))
    assert gt.info["autotuned"] == 1 and gt.info["loads_in_flight"] in (8, 16)
    assert gt.info["depth"] == 0 and gt.info["trail_size"] == 0
    w, nz = gt.currtable()
    assert nz == gt.info["words"]  # every tuple valid again after the trials
    gt.close()


def test_copy_state_ablation_gives_the_same_results():
    """copy_state round-trips currTable through host memory around every call
    (the paper's per-call copies); every call must still match the oracle."""
    seen = _large_stream(100_000, calls=120, seed=13, opt=C.make_options(copy_state=1))
    assert seen["delta"] > 0 and seen["reset"] > 0


@pytest.mark.parametrize("grid", [1, 5, 0])
def test_large_stream_grid_sizes(grid):
    _large_stream(60_000, calls=60, seed=12, opt=C.make_options(grid_blocks=grid), depth=12)


def test_global_plan_path():
    """More supports rows than one CTA stages in shared memory: CTA 0 plans for the grid."""
    dom_lo, dom_size = [0, 0, 0], [3000, 1500, 7]
    tup = G.distinct_uniform_tuples(77, dom_lo, dom_size, 30000)
    tup_ret = O.retained_tuples(tup, dom_lo, dom_size)
    gt = GpuTable(dom_lo, dom_size, tup)
    assert gt.info["local_plan"] == 0 and gt.info["rows"] > 4096
    rng = G.Rng(12)
    masks = [np.ones(d, bool) for d in dom_size]
    st, masks = compare_call(gt, tup_ret, masks)
    gt.save()
    for k in range(8):
        gt.save()
        new, _ = (G.reset_step if k % 2 else G.delta_step)(rng, masks)
        st, out = compare_call(gt, tup_ret, new)
        if st != O.OK:
            gt.restore(0)
            gt.save()
            continue
        masks = out
    gt.close()


@pytest.mark.parametrize("no_early", [0, 1])
def test_filter_beside_the_update_and_after_it(no_early):
    """The default filters calls of few rows beside the update, each probed
    chunk recomputed from the call's rows; with no_early_filter every call
    filters after the update's barrier. Both match the oracle call by call."""
    seen = _large_stream(100_000, calls=160, seed=23, opt=C.make_options(no_early_filter=no_early))
    assert seen["delta"] > 0 and seen["reset"] > 0
    if no_early:
        assert seen["early"] == 0
    else:
        # (most calls of this stream OR at most 16 rows and start from a
        # dense currTable)
        assert 0 < seen["early"] <= seen["calls"]


@pytest.mark.parametrize("grid", [1, 3, 40])
def test_filter_beside_the_update_small_grids(grid):
    # few warps: the probes run on the warps that also update
    seen = _large_stream(30_000, calls=80, seed=29, opt=C.make_options(grid_blocks=grid), depth=10)
    assert seen["early"] > 0


def test_large_stream_1e6_sampled():
    _large_stream(1_000_000, calls=40, seed=13, check_every=4)


# --------------------------------------------------------------------------
# ragged sizes, degenerate inputs
# --------------------------------------------------------------------------

@pytest.mark.parametrize("t", [1, 2, 31, 32, 33, 127, 128, 129, 4095, 4096, 4097, 12345])
def test_ragged_tuple_counts(t):
    dom_lo, dom_size = [3, -2, 0, 5], [5, 7, 33, 20]
    tup = G.distinct_uniform_tuples(G.derive_seed(t, 5), dom_lo, dom_size, t)
    tup_ret = O.retained_tuples(tup, dom_lo, dom_size)
    gt = GpuTable(dom_lo, dom_size, tup)
    assert gt.info["words"] == (t + 31) // 32
    sup = O.supports_matrix(tup, dom_lo, dom_size)
    for r in [0, 4, 5, 11, 12, 44, 45, 46]:
        st, row = C.ct_get_support_row(gt.h, r, gt.info["words"])
        assert row.tolist() == O.pack_words(sup[r]).tolist()
    rng = G.Rng(t)
    masks = [np.ones(d, bool) for d in dom_size]
    gt.save()
    for k in range(12):
        gt.save()
        new, _ = G.remove_random_values(rng, masks, 1 + rng.int(3))
        st, out = compare_call(gt, tup_ret, new)
        if st == O.INFEASIBLE:
            gt.restore(0)
            gt.save()
            masks = [np.ones(d, bool) for d in dom_size]
        else:
            masks = out
    gt.close()


def test_out_of_domain_and_duplicate_tuples():
    dom_lo, dom_size = [0, 0], [4, 4]
    tup = np.array([[0, 0], [4, 1], [1, 1], [1, 1], [-1, 3], [3, 2], [2, 9]], dtype=np.int32)
    tup_ret = O.retained_tuples(tup, dom_lo, dom_size)
    gt = GpuTable(dom_lo, dom_size, tup)
    assert gt.info["tuples"] == len(tup_ret) == 4
    st, out = compare_call(gt, tup_ret, [np.ones(4, bool), np.ones(4, bool)])
    assert st == O.OK
    out[0][0] = False  # domains passed next must be subsets of the last output
    compare_call(gt, tup_ret, out)
    gt.close()


def test_empty_table_is_infeasible():
    for tup in [np.zeros((0, 2), np.int32), np.array([[7, 7]], np.int32)]:
        gt = GpuTable([0, 0], [3, 3], tup)
        assert gt.create_status == C.CT_INFEASIBLE
        st, _, _ = gt.propagate([np.ones(3, bool), np.ones(3, bool)])
        assert st == C.CT_INFEASIBLE
        gt.close()


def test_empty_domain_and_single_values():
    dom_lo, dom_size, tup = G.tiny_table(seed=4)
    tup_ret = O.retained_tuples(tup, dom_lo, dom_size)
    gt = GpuTable(dom_lo, dom_size, tup)
    lv = gt.save()
    st, _, _ = gt.propagate([np.zeros(8, bool), np.ones(8, bool), np.ones(8, bool)])
    assert st == C.CT_INFEASIBLE
    gt.restore(lv)
    lv = gt.save()
    # a full assignment: feasible iff it is a tuple
    row = tup_ret[0]
    masks = [np.eye(8, dtype=bool)[row[i]] for i in range(3)]
    st, _ = compare_call(gt, tup_ret, masks)
    assert st == O.OK
    gt.restore(lv)
    gt.close()


def test_arity_one_and_wide_domains():
    # arity 1: GAC keeps exactly the listed values
    gt = GpuTable([10], [300], np.array([[10], [77], [309], [200], [77]], np.int32))
    tup_ret = O.retained_tuples(gt.tuples, [10], [300])
    compare_call(gt, tup_ret, [np.ones(300, bool)])
    gt.close()
    dom_lo, dom_size = [0, 100, -50], [1000, 70, 129]
    tup = G.distinct_uniform_tuples(9, dom_lo, dom_size, 20000)
    tup_ret = O.retained_tuples(tup, dom_lo, dom_size)
    gt = GpuTable(dom_lo, dom_size, tup)
    rng = G.Rng(3)
    masks = [np.ones(d, bool) for d in dom_size]
    for k in range(10):
        new, _ = G.remove_random_values(rng, masks, 40)
        st, out = compare_call(gt, tup_ret, new)
        if st != O.OK:
            break
        masks = out
    gt.close()


# --------------------------------------------------------------------------
# save / restore, errors
# --------------------------------------------------------------------------

def test_save_restore_round_trip_bit_identical():
    dom_lo, dom_size, tup = G.large_table(21, 50_000)
    tup_ret = O.retained_tuples(tup, dom_lo, dom_size)
    gt = GpuTable(dom_lo, dom_size, tup)
    rng = G.Rng(5)
    masks = [np.ones(d, bool) for d in dom_size]
    snaps = []
    for k in range(6):
        lv = gt.save()
        w, _ = gt.currtable()
        snaps.append((lv, w.copy(), sorted(gt.index().tolist()), [m.copy() for m in masks]))
        new, _ = G.reset_step(rng, masks)
        st, out = compare_call(gt, tup_ret, new)
        assert st == O.OK
        masks = out
    # restore two levels at a time, check bit identity, then continue from there
    for lv, w0, idx0, m0 in reversed(snaps[::2]):
        gt.restore(lv)
        w, _ = gt.currtable()
        assert np.array_equal(w, w0)
        assert sorted(gt.index().tolist()) == idx0
        # lastDom restored too: propagating the saved domains changes nothing in currTable
        st, out = compare_call(gt, tup_ret, m0)
        assert st == O.OK
        gt.save()
        gt.restore(lv)
    gt.close()


def test_error_codes():
    dom_lo, dom_size, tup = G.tiny_table(seed=6)
    gt = GpuTable(dom_lo, dom_size, tup)
    assert C.ct_restore(gt.h, 0) == C.CT_ERR_LEVEL
    lv = gt.save()
    m = [np.ones(8, bool) for _ in range(3)]
    m[0][:4] = False
    st, _, _ = gt.propagate(m)
    assert st in (C.CT_OK, C.CT_INFEASIBLE)
    if st == C.CT_OK:
        # growing a domain without restore
        st, _, _ = gt.propagate([np.ones(8, bool) for _ in range(3)])
        assert st == C.CT_ERR_STATE
        assert "grew" in C.last_error()
    gt.restore(lv)
    lv = gt.save()
    st, _, _ = gt.propagate([np.zeros(8, bool), np.ones(8, bool), np.ones(8, bool)])
    assert st == C.CT_INFEASIBLE
    st, _, _ = gt.propagate([np.ones(8, bool) for _ in range(3)])
    assert st == C.CT_ERR_STATE
    gt.restore(lv)
    st, _, _ = gt.propagate([np.ones(8, bool) for _ in range(3)])
    assert st == C.CT_OK
    assert C.ct_restore(gt.h, 5) == C.CT_ERR_LEVEL
    gt.close()


def test_host_buffer_entry_point_matches_device_entry_point():
    dom_lo, dom_size, tup = G.large_table(31, 20_000)
    tup_ret = O.retained_tuples(tup, dom_lo, dom_size)
    gt = GpuTable(dom_lo, dom_size, tup)
    rng = G.Rng(8)
    masks = [np.ones(d, bool) for d in dom_size]
    for k in range(10):
        new, _ = G.reset_step(rng, masks) if k % 2 else G.delta_step(rng, masks)
        words = C.masks_to_words(new)
        st, ch = C.ct_propagate_host(gt.h, words, gt.nch)
        st_o, out_o, _ = oracle_step(tup_ret, dom_lo, new)
        assert st == st_o
        if st != O.OK:
            break
        got = C.words_to_masks(words, dom_size)
        for i in range(6):
            assert np.array_equal(got[i], out_o[i])
        masks = out_o
    gt.close()


@pytest.mark.parametrize("arity,d,t", [(6, 32, 20_000), (3, 1000, 5_000)])
def test_host_buffer_calls_with_backtracking(arity, d, t):
    """ct_propagate_host over a delta/reset stream with saves, restores and
    wipe-outs: status, domains and changed mask equal the oracle's call by
    call. With 6 words of domains they travel in the launch parameters (up to
    16 words do); with 96 words (d = 1000) they are copied."""
    seed = 7100 + d
    dom_lo, dom_size, tup = G.large_table(seed, t, arity, d)
    tup_ret = O.retained_tuples(tup, dom_lo, dom_size)
    gt = GpuTable(dom_lo, dom_size, tup)
    nch = (arity + 31) // 32
    rng = G.Rng(G.derive_seed(seed, 1))
    root = [np.ones(x, bool) for x in dom_size]
    assert gt.save() == 0
    masks, depth, seen = root, 0, {"ok": 0, "fail": 0, "pruned": 0}
    for k in range(40):
        gt.save()
        new, _ = G.reset_step(rng, masks) if k % 2 else G.delta_step(rng, masks)
        words = C.masks_to_words(new)
        st, ch = C.ct_propagate_host(gt.h, words, nch)
        st_o, out_o, _ = oracle_step(tup_ret, dom_lo, new)
        assert st == st_o, (k, C.last_error())
        depth += 1
        if st != O.OK:
            seen["fail"] += 1
            gt.restore(1)  # the dive's first save: the root state (level 0 stays)
            masks, depth = root, 0
            continue
        seen["ok"] += 1
        got = C.words_to_masks(words, dom_size)
        changed = 0
        for i in range(arity):
            assert np.array_equal(got[i], out_o[i]), (k, i)
            if not np.array_equal(out_o[i], new[i]):
                changed |= 1 << i
        assert int(ch[0]) == changed, k
        seen["pruned"] += changed != 0
        masks = out_o
        if depth >= 8:
            gt.restore(1)
            masks, depth = root, 0
    # a grown domain is refused on the host path as on the device path
    gt.restore(0)
    gt.save()
    cut = [m.copy() for m in root]
    cut[0][np.flatnonzero(cut[0])[1:]] = False
    st, _ = C.ct_propagate_host(gt.h, C.masks_to_words(cut), nch)
    assert st in (C.CT_OK, C.CT_INFEASIBLE)
    if st == C.CT_OK:
        st, _ = C.ct_propagate_host(gt.h, C.masks_to_words(root), nch)
        assert st == C.CT_ERR_STATE
    assert seen["ok"] > 0 and seen["pruned"] > 0, seen
    gt.close()


def test_profiling_switched_on_and_off():
    """ct_set_profile: calls are timed only while profiling is on; results
    are the oracle's either way."""
    dom_lo, dom_size, tup = G.large_table(33, 20_000)
    tup_ret = O.retained_tuples(tup, dom_lo, dom_size)
    gt = GpuTable(dom_lo, dom_size, tup)
    rng = G.Rng(9)
    masks = [np.ones(d, bool) for d in dom_size]
    timed = []
    for k in range(6):
        assert C.ct_set_profile(gt.h, k % 2) == C.CT_OK
        new, _ = G.delta_step(rng, masks)
        st, out, _ = gt.propagate(new)
        timed.append(k % 2)
        st_o, out_o, _ = oracle_step(tup_ret, dom_lo, new)
        assert st == st_o
        if st != O.OK:
            break
        assert all(np.array_equal(a, b) for a, b in zip(out, out_o))
        masks = out_o
    st, prof = C.ct_get_profile(gt.h)
    assert st == C.CT_OK and prof["calls"] == sum(timed) and prof["kernel_ms"] > 0
    gt.close()


# --------------------------------------------------------------------------
# full-size workloads, sampled against the oracle
# --------------------------------------------------------------------------

def test_bench_size_4e6_sampled():
    _large_stream(4_000_000, calls=12, seed=41, check_every=3, depth=6)


def test_huge_1e7_arity5_sampled():
    dom_lo, dom_size, tup = G.large_table(51, 10_000_000, arity=5, d=64)
    tup_ret = O.retained_tuples(tup, dom_lo, dom_size)
    gt = GpuTable(dom_lo, dom_size, tup)
    assert gt.info["rows"] == 320
    rng = G.Rng(9)
    masks = [np.ones(d, bool) for d in dom_size]
    st, masks = compare_call(gt, tup_ret, masks)
    gt.save()
    for k in range(4):
        gt.save()
        new, _ = G.reset_step(rng, masks)
        st, out = compare_call(gt, tup_ret, new, check_table=(k == 3))
        if st != O.OK:
            break
        masks = out
    # delta calls on the table of more segments than one wave of warps (8
    # loads per batch): filtered beside the update
    assert st == O.OK
    early = 0
    for k in range(2):
        gt.save()
        new, i = G.delta_step(rng, masks)
        if i is None:
            break
        st, out = compare_call(gt, tup_ret, new, check_table=(k == 1))
        early += gt.stats()["early_filter"]
        if st != O.OK:
            break
        masks = out
    assert early > 0
    gt.close()


def test_read_ceiling_entry_point():
    """The measurement kernel reads a device buffer and rejects what it cannot read."""
    torch = torch_cuda()
    C.load()
    x = torch.ones(1 << 20, dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream()
    assert C.ct_read_ceiling(x, x.numel() * 4, s) == C.CT_OK
    assert C.ct_read_ceiling(x, 16, s) == C.CT_OK
    st, ms = C.ct_read_ceiling(x, x.numel() * 4, s, timed=True)
    assert st == C.CT_OK and 0.0 < ms < 1000.0
    torch.cuda.synchronize()
    assert C.ct_read_ceiling(x, 0, s) == C.CT_ERR_ARG
    assert C.ct_read_ceiling(x, 24, s) == C.CT_ERR_ARG
    assert C.ct_read_ceiling(x.data_ptr() + 4, 16, s) == C.CT_ERR_ARG
    assert C.ct_read_ceiling(0, 16, s) == C.CT_ERR_ARG
