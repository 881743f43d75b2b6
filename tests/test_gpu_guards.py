"""Device-buffer checks that need no sanitizer (the library's ct_debug_* test
hooks): guard regions around every buffer a table owns stay untouched through
streams of propagations, saves and restores (no kernel writes outside its
buffers, the trail and the level stack included), and a table creation that
runs out of device memory at any of its allocations returns CT_ERR_OOM and
gives back every byte it took."""
import gc

import numpy as np
import pytest

from oracle import ct_oracle as O
from oracle import short as S
from paper_2507_18413_gb300 import ct as C
from paper_2507_18413_gb300 import inputs as G
from gpu_helpers import GpuTable, compare_call, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture
def guarded():
    torch_cuda()
    C.load()
    assert C.ct_debug_guard_buffers(1) == C.CT_OK
    yield
    C.ct_debug_guard_buffers(0)


def _dives(gt, call, root, seed, calls, depth):
    """Delta/reset edits in dives from the root, restored after a failure or
    `depth` calls; `call(masks)` checks one call and returns (status, out)."""
    rng = G.Rng(seed)
    gt.save()
    masks, d, fails = root, 0, 0
    for _ in range(calls):
        gt.save()
        new, i = (G.delta_step if rng.int(2) == 0 else G.reset_step)(rng, masks)
        if i is None:
            new, _ = G.remove_random_values(rng, masks, 1)
        st, out = call(new)
        d += 1
        if st == O.INFEASIBLE or d >= depth:
            fails += st == O.INFEASIBLE
            gt.restore(0)
            gt.save()
            masks, d = root, 0
        else:
            masks = out
    return fails


def _guards_intact(gt):
    st, changed = C.ct_debug_check_guards(gt.h)
    assert st == C.CT_OK, C.last_error()
    assert changed == 0, f"{changed} guard bytes changed"


@pytest.mark.parametrize("t,opt", [(100_000, {}), (100_000, {"no_early_filter": 1}), (60_000, {"grid_blocks": 3}),
                                   (30_000, {"no_split": 1, "no_residues": 1})])
def test_no_write_outside_the_buffers_on_streams(guarded, t, opt):
    seed = 91 + t
    dom_lo, dom_size, tup = G.large_table(seed, t)
    ret = O.retained_tuples(tup, dom_lo, dom_size)
    gt = GpuTable(dom_lo, dom_size, tup, opt=C.make_options(**opt))
    st, root = compare_call(gt, ret, [np.ones(d, bool) for d in dom_size])
    assert st == O.OK
    _dives(gt, lambda m: compare_call(gt, ret, m, check_table=False), root, seed, calls=120, depth=10)
    _guards_intact(gt)
    gt.close()


def test_no_write_outside_the_buffers_short_table(guarded):
    seed, arity, d = 4321, 4, 24
    dom_lo, dom_size = [0] * arity, [d] * arity
    tup = G.short_tuples(seed, dom_lo, dom_size, G.cap_distinct(dom_size, 60_000), star_prob=0.1)
    ret = S.retained_short(tup, dom_lo, dom_size)
    gt = GpuTable(dom_lo, dom_size, tup)

    def call(masks):
        st_o, out_o, _ = S.gac_table_short(ret, dom_lo, masks)
        st_g, out_g, _ = gt.propagate(masks)
        assert st_g == st_o
        if st_o == O.OK:
            for i in range(arity):
                assert np.array_equal(out_g[i], out_o[i])
        return st_o, out_o

    st, root = call([np.ones(x, bool) for x in dom_size])
    assert st == O.OK
    _dives(gt, call, root, seed, calls=60, depth=6)
    _guards_intact(gt)
    gt.close()


def test_the_guard_check_sees_a_changed_guard(guarded):
    dom_lo, dom_size, tup = G.large_table(5, 4_000)
    gt = GpuTable(dom_lo, dom_size, tup)
    _guards_intact(gt)
    st, changed = C.ct_debug_check_guards(gt.h, poke=3)
    assert st == C.CT_OK and changed == 3
    st, changed = C.ct_debug_check_guards(gt.h)
    assert changed == 3  # the guard stays as it was left
    assert C.ct_debug_check_guards(gt.h, poke=257)[0] == C.CT_ERR_ARG
    gt.close()


def test_unguarded_tables_report_no_guards():
    torch_cuda()
    C.load()
    dom_lo, dom_size, tup = G.large_table(6, 2_000)
    gt = GpuTable(dom_lo, dom_size, tup)
    assert C.ct_debug_check_guards(gt.h, poke=5) == (C.CT_OK, 0)
    gt.close()


def test_failed_allocations_give_back_every_byte():
    """Every allocation of ct_create made to fail in turn: each creation returns
    CT_ERR_OOM with the library's device bytes back at their count before it,
    and the creation that gets all its buffers gives a table that propagates
    and, destroyed, returns them too."""
    torch_cuda()
    C.load()
    dom_lo, dom_size, tup = G.large_table(77, 20_000)
    ret = O.retained_tuples(tup, dom_lo, dom_size)
    gc.collect()  # tables of earlier tests left to the collector give their bytes back first
    st, base = C.ct_debug_device_bytes()
    assert st == C.CT_OK
    n = 0
    try:
        while True:
            C.ct_debug_fail_alloc(n)
            st, h = C.ct_create(len(dom_lo), dom_lo, dom_size, tup)
            if st >= 0:
                break
            assert st == C.CT_ERR_OOM, (n, st, C.last_error())
            assert C.ct_debug_device_bytes()[1] == base, f"allocation {n} failed: bytes not given back"
            n += 1
            assert n < 100
    finally:
        C.ct_debug_fail_alloc(-1)
    assert n >= 10  # the buffers of a table
    assert C.ct_debug_device_bytes()[1] > base
    C.ct_destroy(h)
    assert C.ct_debug_device_bytes()[1] == base
    # and a table created normally after it works
    gt = GpuTable(dom_lo, dom_size, tup)
    st, _ = compare_call(gt, ret, [np.ones(d, bool) for d in dom_size])
    assert st == O.OK
    gt.close()
    assert C.ct_debug_device_bytes()[1] == base
