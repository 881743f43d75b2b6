"""Pins of the short-table oracle (oracle/short.py): a short table must filter
exactly like the ground table it stands for, and hand-checked cases."""
import numpy as np

from oracle import ct_oracle as O
from oracle import short as S
from paper_2507_18413_gb300 import inputs as G


def test_short_table_filters_like_its_expansion():
    rng = np.random.default_rng(11)
    for trial in range(60):
        arity = int(rng.integers(1, 4))
        sizes = [int(v) for v in rng.integers(1, 5, size=arity)]
        lo = [int(v) for v in rng.integers(-2, 3, size=arity)]
        tup = G.short_tuples(int(rng.integers(1 << 30)), lo, sizes, G.cap_distinct(sizes, 6), star_prob=0.3)
        ret = S.retained_short(tup, lo, sizes)
        ground = O.retained_tuples(S.expand(ret, lo, sizes), lo, sizes)
        masks = [rng.random(d) < 0.7 for d in sizes]
        for m in masks:  # propagation never sees an empty domain (it fails first)
            if not m.any():
                m[int(rng.integers(len(m)))] = True
        st, out, valid = S.gac_table_short(ret, lo, masks)
        if len(ground) == 0:
            assert st == O.INFEASIBLE
            continue
        st_g, out_g, _ = O.gac_table(ground, lo, masks)
        assert st == st_g
        if st == O.OK:
            for a, b in zip(out, out_g):
                assert np.array_equal(a, b)
        # a short tuple is valid iff one of its expansions is
        for j, t in enumerate(ret):
            e = S.expand(t[None, :], lo, sizes)
            assert valid[j] == bool(O.valid_mask(e, lo, masks).any())


def test_short_table_hand_cases():
    # (1, *) over {0,1} x {0,1}: x0 = 1 only, x1 untouched
    tup = np.array([[1, S.STAR]])
    st, out, valid = S.gac_table_short(tup, [0, 0], [np.ones(2, bool), np.ones(2, bool)])
    assert st == O.OK and out[0].tolist() == [False, True] and out[1].tolist() == [True, True]
    # (*, *) supports everything, even after x0 lost a value
    tup = np.array([[S.STAR, S.STAR]])
    st, out, _ = S.gac_table_short(tup, [0, 0], [np.array([True, False]), np.ones(2, bool)])
    assert st == O.OK and out[0].tolist() == [True, False] and out[1].tolist() == [True, True]
    # (0, *) and (*, 2): removing x0 = 0 leaves only (*, 2) -> x1 = 2
    tup = np.array([[0, S.STAR], [S.STAR, 2]])
    st, out, valid = S.gac_table_short(tup, [0, 0], [np.array([False, True]), np.ones(3, bool)])
    assert st == O.OK and valid.tolist() == [False, True] and out[1].tolist() == [False, False, True]
    # a component outside the initial domain drops the tuple; wildcards never do
    ret = S.retained_short(np.array([[5, S.STAR], [S.STAR, 1]]), [0, 0], [2, 2])
    assert ret.tolist() == [[S.STAR, 1]]


def test_short_tuples_generator():
    t = G.short_tuples(3, [0, 0, 0], [4, 4, 4], 20, star_prob=0.25)
    assert t.shape == (20, 3) and (t == S.STAR).any() and ((t == S.STAR) | ((t >= 0) & (t < 4))).all()
