"""Bounded device waits, exercised without a fault or a hang.

Every grid-barrier wait of the propagation kernel gives up after a number of
polls, records CT_ERR_TIMEOUT and returns. ct_arm_wait_timeout sets the next
call's barrier count where no CTA can complete it and makes the poll limit
small, so every wait of that call runs out quickly; the kernel then exits
without publishing, the host maps that to CT_ERR_TIMEOUT, the table refuses
later calls, and the context stays usable (a new table on the same stream
matches the oracle).
"""
import numpy as np
import pytest

from oracle import ct_oracle as O
from paper_2507_18413_gb300 import ct as C
from paper_2507_18413_gb300 import inputs as G
from gpu_helpers import GpuTable, compare_call, torch_cuda

pytestmark = pytest.mark.gpu


def test_barrier_wait_runs_out_and_the_table_refuses_later_calls():
    torch_cuda()
    dom_lo, dom_size, tup = G.large_table(5, 50_000)
    tup_ret = O.retained_tuples(tup, dom_lo, dom_size)
    gt = GpuTable(dom_lo, dom_size, tup)
    rng = G.Rng(4)
    st, root = compare_call(gt, tup_ret, [np.ones(d, bool) for d in dom_size])
    assert st == O.OK
    gt.save()
    assert C.ct_arm_wait_timeout(gt.h, 0) == C.CT_ERR_ARG
    assert C.ct_arm_wait_timeout(gt.h, 2000) == C.CT_OK
    new, _ = G.reset_step(rng, root)
    st, _, _ = gt.propagate(new)
    assert st == C.CT_ERR_TIMEOUT, (st, C.last_error())
    assert "wait ran out" in C.last_error()
    # the table is unusable from here on
    st, _ = C.ct_propagate(gt.h, gt.dom, 1)
    assert st == C.CT_ERR_TIMEOUT
    assert C.ct_restore(gt.h, 0) == C.CT_ERR_TIMEOUT
    gt.close()
    # the device and the stream still work: a new table matches the oracle
    gt2 = GpuTable(dom_lo, dom_size, tup)
    st, masks = compare_call(gt2, tup_ret, [np.ones(d, bool) for d in dom_size])
    gt2.save()
    for k in range(6):
        gt2.save()
        new, _ = (G.delta_step if k % 2 else G.reset_step)(rng, masks)
        st, out = compare_call(gt2, tup_ret, new)
        if st != O.OK:
            gt2.restore(0)
            gt2.save()
            continue
        masks = out
    gt2.close()
