"""Pins of the negative-table oracle (oracle/negative.py) against brute force:
a negative table filters exactly like the positive table of its allowed tuples."""
import itertools

import numpy as np

from oracle import ct_oracle as O
from oracle import negative as N


def test_negative_table_filters_like_its_complement():
    rng = np.random.default_rng(21)
    for trial in range(80):
        arity = int(rng.integers(1, 4))
        sizes = [int(v) for v in rng.integers(1, 5, size=arity)]
        lo = [int(v) for v in rng.integers(-1, 2, size=arity)]
        space = list(itertools.product(*[range(l, l + s) for l, s in zip(lo, sizes)]))
        forb = [list(c) for c in space if rng.random() < 0.6] or [list(space[0])]
        forb += forb[: int(rng.integers(0, 3))]          # duplicates count once
        tup = N.retained_negative(forb, lo, sizes)
        allowed = N.complement(tup, lo, sizes)
        masks = [rng.random(d) < 0.7 for d in sizes]
        for m in masks:
            if not m.any():
                m[int(rng.integers(len(m)))] = True
        st, out, valid = N.gac_table_negative(tup, lo, masks)
        if len(allowed) == 0:
            assert st == O.INFEASIBLE
            continue
        st_p, out_p, _ = O.gac_table(allowed, lo, masks)
        assert st == st_p
        if st == O.OK:
            for a, b in zip(out, out_p):
                assert np.array_equal(a, b)


def test_negative_hand_cases():
    # forbid (0,0) and (0,1) over {0,1}^2: x0 = 0 has no allowed partner
    tup = N.retained_negative([[0, 0], [0, 1], [0, 1]], [0, 0], [2, 2])
    assert len(tup) == 2
    st, out, valid = N.gac_table_negative(tup, [0, 0], [np.ones(2, bool), np.ones(2, bool)])
    assert st == O.OK and out[0].tolist() == [False, True] and out[1].tolist() == [True, True]
    # with x1 = {1} only, x0 = 1 stays (tuple (1,1) allowed)
    st, out, _ = N.gac_table_negative(tup, [0, 0], [np.ones(2, bool), np.array([False, True])])
    assert st == O.OK and out[0].tolist() == [False, True]
    # nothing valid forbidden: everything stays
    st, out, valid = N.gac_table_negative(tup, [0, 0], [np.array([False, True]), np.ones(2, bool)])
    assert st == O.OK and not valid.any() and out[1].tolist() == [True, True]
    # every combination forbidden: infeasible
    allf = N.retained_negative([[0, 0], [0, 1], [1, 0], [1, 1]], [0, 0], [2, 2])
    st, _, _ = N.gac_table_negative(allf, [0, 0], [np.ones(2, bool), np.ones(2, bool)])
    assert st == O.INFEASIBLE
