"""GPU parity of updateTable with a segment's row list cut over several warps.

Algorithm 2 ANDs one mask per changed variable into currTable, each the OR of
that variable's rows (complemented on the delta path). The kernel cuts a call's
row list into G = 1, 2, 4 or 8 slices per 32-chunk segment (one batch of row
loads per slice where the list allows) and combines the slices in row order,
so a variable's rows may be split between warps, or fill a slice without
beginning or ending in it. Every call here is compared bit-exactly with the
oracle (status, domains, changed mask, currTable words, the non-zero index)
and with the same calls on a table created with ct_options.no_split = 1 (one
warp walks the whole list), on row counts that take every G, cuts inside a
variable, and mix delta-path and reset-path variables.
"""
import numpy as np
import pytest

from oracle import ct_oracle as O
from oracle import short as S
from paper_2507_18413_gb300 import ct as C
from paper_2507_18413_gb300 import inputs as G
from gpu_helpers import GpuTable, compare_call, torch_cuda

pytestmark = pytest.mark.gpu


def _mixed_edit(rng, masks, nvars_changed, heavy=False):
    """Reduce `nvars_changed` random variables: each on the delta path (fewer
    values removed than kept) or on the reset path (more removed than kept).
    heavy: the most rows each path allows (just under half removed, or half kept)."""
    new = [m.copy() for m in masks]
    order = np.argsort(rng.u64(len(masks)), kind="stable")[:nvars_changed]
    for i in order:
        vals = np.flatnonzero(new[i])
        if len(vals) < 2:
            continue
        if rng.int(2) == 0:
            # delta: |removed| < |kept|
            k = (len(vals) - 1) // 2 if heavy else 1 + rng.int(max(1, (len(vals) - 1) // 2))
        else:
            # reset: |removed| >= |kept|
            k = len(vals) - len(vals) // 2 if heavy else \
                len(vals) // 2 + 1 + rng.int(max(1, len(vals) - len(vals) // 2 - 1))
        k = max(1, min(k, len(vals) - 1))
        drop = vals[np.argsort(rng.u64(len(vals)), kind="stable")[:k]]
        new[i][drop] = False
    return new


def _rows_of(stats):
    return stats["rows_ored"]


def _slices(rows, U=16, maxG=8):
    g = 1
    while g < maxG and g < (rows + U - 1) // U:
        g *= 2
    return g


@pytest.mark.parametrize("t,seed", [(200_000, 3), (70_001, 4)])
def test_split_update_matches_oracle_and_unsplit(t, seed):
    torch_cuda()
    dom_lo, dom_size, tup = G.large_table(seed, t)
    tup_ret = O.retained_tuples(tup, dom_lo, dom_size)
    a = GpuTable(dom_lo, dom_size, tup)
    b = GpuTable(dom_lo, dom_size, tup, opt=C.make_options(no_split=1))
    rng = G.Rng(G.derive_seed(seed, 9))
    root = [np.ones(d, bool) for d in dom_size]
    st, root = compare_call(a, tup_ret, root)
    st_b, out_b, _ = b.propagate([np.ones(d, bool) for d in dom_size])
    assert st == st_b == O.OK
    a.save()
    b.save()
    seen = set()
    for k in range(60):
        masks = root
        depth = 1 + rng.int(3)
        for d in range(depth):
            a.save()
            b.save()
            heavy = d == 0 and k % 4 == 0
            new = _mixed_edit(rng, masks, 6 if heavy else 1 + rng.int(6), heavy=heavy)
            st, out = compare_call(a, tup_ret, new)
            s = a.stats()
            seen.add(_slices(_rows_of(s)))
            st_b, out_b, _ = b.propagate(new)
            assert st_b == st
            if st != O.OK:
                break
            for i in range(6):
                assert np.array_equal(out_b[i], out[i])
            assert np.array_equal(b.currtable()[0], a.currtable()[0])
            masks = out
        a.restore(0)
        b.restore(0)
        a.save()
        b.save()
    # the streams took several slice counts, including a cut over 8 warps
    assert {1, 8} <= seen and len(seen) >= 3, seen
    a.close()
    b.close()


def test_split_short_table_delta_rows():
    """Short tables OR different rows on the delta path (without the wildcards):
    the split must keep each slice's rows on the right row set."""
    torch_cuda()
    arity, d, seed = 5, 24, 71
    dom_lo, dom_size = [0] * arity, [d] * arity
    tup = G.short_tuples(seed, dom_lo, dom_size, 60_000, star_prob=0.15)
    ret = S.retained_short(tup, dom_lo, dom_size)
    gt = GpuTable(dom_lo, dom_size, tup)
    rng = G.Rng(3)
    root = [np.ones(x, bool) for x in dom_size]
    st_o, root, _ = S.gac_table_short(ret, dom_lo, root)
    st_g, out_g, _ = gt.propagate([np.ones(x, bool) for x in dom_size])
    assert st_g == st_o == O.OK
    gt.save()
    for k in range(25):
        gt.save()
        new = _mixed_edit(rng, root, 2 + rng.int(4))
        st_o, out_o, valid = S.gac_table_short(ret, dom_lo, new)
        st_g, out_g, _ = gt.propagate(new)
        assert st_g == st_o
        if st_o == O.OK:
            for i in range(arity):
                assert np.array_equal(out_g[i], out_o[i])
            assert np.array_equal(gt.currtable()[0], O.currtable_words(valid))
        gt.restore(0)
        gt.save()
    gt.close()


def test_split_global_plan_long_row_lists():
    """More rows than a CTA stages in shared memory (codes beyond 4,096 are read
    from global memory) and slices of hundreds of rows."""
    torch_cuda()
    dom_lo, dom_size = [0, 0, 0], [6000, 3000, 7]
    tup = G.distinct_uniform_tuples(78, dom_lo, dom_size, 40000)
    tup_ret = O.retained_tuples(tup, dom_lo, dom_size)
    gt = GpuTable(dom_lo, dom_size, tup)
    assert gt.info["local_plan"] == 0
    masks = [np.ones(d, bool) for d in dom_size]
    st, root = compare_call(gt, tup_ret, masks)
    gt.save()
    rng = G.Rng(5)
    rows = []
    for k in range(6):
        gt.save()
        new = [m.copy() for m in root]
        for i in (0, 1):
            vals = np.flatnonzero(new[i])
            # even k: reset path (a third kept); odd k: delta path (just under half removed)
            keep = len(vals) // 3 if k % 2 == 0 else len(vals) - (len(vals) - 1) // 2
            drop = vals[np.argsort(rng.u64(len(vals)), kind="stable")[keep:]]
            new[i][drop] = False
        st, out = compare_call(gt, tup_ret, new)
        rows.append(gt.stats()["rows_ored"])
        gt.restore(0)
        gt.save()
    assert max(rows) > 4096, rows
    gt.close()
