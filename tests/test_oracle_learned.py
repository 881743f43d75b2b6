"""Pins of the learned-order oracle (oracle/learned.py) against closed forms,
hand counts, finite differences and brute force; CPU only."""
import json
import math
import os

import numpy as np

from oracle import ct_oracle as O
from oracle import learned as L
from paper_2507_18413_gb300 import inputs as G


def _table1(golden_dir):
    with open(os.path.join(golden_dir, "table1.json")) as f:
        g = json.load(f)
    csp = O.Csp(g["scope_dom_lo"], g["scope_dom_size"])
    csp.add_table([0, 1, 2], g["tuples"]["rows"])
    return csp, g


def test_feature_closed_form_on_a_full_product_table():
    """Every combination allowed: p_c(a) = 1/s for every value, so bal = 1,
    top = 1/s, normalised entropy = 1, live = product of the sizes."""
    import itertools
    sizes = [3, 4, 5]
    rows = [list(t) for t in itertools.product(*[range(d) for d in sizes])]
    csp = O.Csp([0, 0, 0], sizes)
    csp.add_table([0, 1, 2], rows)
    F = L.features(csp, csp.full_masks())
    for x, s in enumerate(sizes):
        assert F[x, 0] == 1.0
        assert math.isclose(F[x, 1], math.log2(s) / 8)
        assert F[x, 2] == 1.0
        assert math.isclose(F[x, 3], 1.0)
        assert math.isclose(F[x, 4], 1.0 / s)
        assert math.isclose(F[x, 5], 1.0)
        assert math.isclose(F[x, 6], math.log2(1 + 60) / 32)
        assert math.isclose(F[x, 7], s / 5)


def test_features_by_hand_on_table1(golden_dir):
    """The paper's worked example (Table 1): 5 tuples over x1, x2, x3, domains
    {1..4}. At its GAC fixpoint (read off by hand: x1 = 4 and x3 in {2, 4} have
    no tuple) all 5 tuples are valid, and the value counts are
    x1: 1->2, 2->1, 3->2;  x2: 1,2,3->1, 4->2;  x3: 1->2, 3->3."""
    csp, g = _table1(golden_dir)
    assert len(g["tuples"]["rows"]) == 5
    masks = [np.array([1, 1, 1, 0], bool), np.ones(4, bool), np.array([1, 0, 1, 0], bool)]
    F = L.features(csp, masks)
    for x, cnt, s in ((0, [2, 1, 2], 3), (1, [1, 1, 1, 2], 4), (2, [2, 3], 2)):
        p = np.array(cnt) / 5
        assert math.isclose(F[x, 0], s / 4)
        assert math.isclose(F[x, 3], s * p.min())
        assert math.isclose(F[x, 4], p.max())
        assert math.isclose(F[x, 5], -(p * np.log2(p)).sum() / math.log2(s))
        assert math.isclose(F[x, 6], math.log2(6) / 32)
        assert math.isclose(F[x, 7], s / 4)
    assert math.isclose(F[0, 3], 0.6) and math.isclose(F[1, 3], 0.8) and math.isclose(F[2, 4], 0.6)


def test_features_with_a_valid_tuple_filter_brute_force():
    """Random small tables and random domains: counts of valid tuples per value
    recomputed by enumerating the product of the current domains and testing
    membership in the tuple set."""
    import itertools
    rng = np.random.default_rng(3)
    for trial in range(20):
        sizes = [int(v) for v in rng.integers(2, 5, size=4)]
        csp = O.Csp([0] * 4, sizes)
        tabs = []
        for _ in range(3):
            sc = [int(v) for v in rng.choice(4, size=2 + int(rng.integers(0, 2)), replace=False)]
            allt = list(itertools.product(*[range(sizes[v]) for v in sc]))
            keep = [list(t) for t in allt if rng.random() < 0.6] or [list(allt[0])]
            csp.add_table(sc, keep)
            tabs.append((sc, set(map(tuple, keep))))
        masks = [rng.random(d) < 0.8 for d in sizes]
        for m in masks:
            if m.sum() == 0:
                m[0] = True
        F = L.features(csp, masks)
        sizes_now = [int(m.sum()) for m in masks]
        for x in range(4):
            if sizes_now[x] < 2:
                assert not F[x].any()
                continue
            bal = []
            for sc, tset in tabs:
                if x not in sc:
                    continue
                combos = list(itertools.product(*[np.flatnonzero(masks[v]) for v in sc]))
                valid = [c for c in combos if tuple(int(a) for a in c) in tset]
                if not valid:
                    continue
                k = sc.index(x)
                cnt = [sum(1 for c in valid if c[k] == a) for a in np.flatnonzero(masks[x])]
                bal.append(sizes_now[x] * min(cnt) / len(valid))
            if bal:
                assert math.isclose(F[x, 3], float(np.mean(bal)), rel_tol=1e-12)
            else:
                assert F[x, 3] == 0.0


def test_forward_closed_form():
    w = np.zeros(L.NW)
    o1 = 0
    ob1 = L.H * L.NF
    o2 = ob1 + L.H
    ob2 = o2 + L.H * L.H
    o3 = ob2 + L.H
    ob3 = o3 + L.H
    w[o1 + 0 * L.NF + 0] = 1.0     # h1[0] = relu(x0)
    w[o2 + 0 * L.H + 0] = 2.0      # h2[0] = relu(2 h1[0])
    w[o3 + 0] = 3.0                # out = 3 h2[0] + b3
    w[ob3] = 0.5
    X = np.zeros((3, L.NF))
    X[:, 0] = [1.0, -1.0, 2.5]
    assert np.allclose(L.forward(w, X), [6.5, 0.5, 15.5])


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(7)
    w = G.mlp_init_weights(11).astype(np.float64)
    w[L.H * L.NF:L.H * L.NF + L.H] = rng.normal(0, 0.1, L.H)  # non-zero b1: both ReLU sides
    X = rng.random((9, L.NF))
    y = rng.random(9)
    loss, g = L.loss_grad(w, X, y)
    h = 1e-6
    idx = rng.choice(L.NW, size=60, replace=False)
    for i in idx:
        wp = w.copy()
        wm = w.copy()
        wp[i] += h
        wm[i] -= h
        lp, _ = L.loss_grad(wp, X, y)
        lm, _ = L.loss_grad(wm, X, y)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    r = L.forward(w, X) - y
    assert math.isclose(loss, float((r * r).sum() / 18))


def test_first_adam_step_moves_each_weight_by_lr():
    """t = 1: the bias-corrected moments are g and g^2, so the step is
    -lr * g / (|g| + eps)."""
    rng = np.random.default_rng(1)
    w = rng.normal(size=L.NW)
    g = rng.normal(size=L.NW)
    w1, m, v = L.adam_step(w, g, np.zeros(L.NW), np.zeros(L.NW), 1, 0.01)
    assert np.allclose(w1 - w, -0.01 * g / (np.abs(g) + L.EPS), rtol=1e-12, atol=0)


def test_training_fits_a_learnable_target():
    rng = np.random.default_rng(5)
    X = rng.random((512, L.NF))
    y = 0.7 * X[:, 0] - 0.3 * X[:, 3] + 0.1
    w0 = G.mlp_init_weights(2)
    perms = G.epoch_orders(9, 512, 30)
    w, losses = L.train(w0, X, y, perms, 64, 3e-3)
    assert losses[-1] < 0.05 * losses[0]
    assert losses[-1] < 1e-3


def test_lookahead_labels_closed_cases():
    # x0 = x1 over {0,1}: fixing x0 fixes x1, the log-size goes 2 -> 0
    csp = O.Csp([0, 0], [2, 2])
    csp.add_table([0, 1], [[0, 0], [1, 1]])
    assert L.lookahead_label(csp, csp.full_masks(), 0) == 1.0
    # free x1: fixing x0 leaves log2|D1| = 1 of 2
    csp = O.Csp([0, 0], [2, 2])
    csp.add_table([0], [[0], [1]])
    assert L.lookahead_label(csp, csp.full_masks(), 0) == 0.5
    # fixing x0 to 0 fails: the only tuples with x0 = 0 need x1 = 2, removed
    csp = O.Csp([0, 0], [2, 3])
    csp.add_table([0, 1], [[0, 2], [1, 0], [1, 1]])
    masks = [np.array([True, True]), np.array([True, True, False])]
    assert L.lookahead_label(csp, masks, 0) == 1.0


def test_learned_policy_searches_the_same_tree_size_when_all_solutions_are_counted():
    """Any branching order visits a tree whose solution count is the CSP's;
    the learned order must find exactly the oracle's solutions."""
    rng = G.Rng(12)
    csp = O.Csp([0] * 6, [4] * 6)
    for k in range(4):
        sc = G.random_scope(rng, 6, 3)
        csp.add_table(sc, G.distinct_uniform_tuples(G.derive_seed(12, k), [0] * 3, [4] * 3, 30))
    w = G.mlp_init_weights(4)
    a = O.dfs(csp)
    b = O.dfs(csp, select=L.select_learned(csp, w))
    assert a.solutions == b.solutions
    # replaying the learned decisions reproduces its tree exactly
    dec = []
    sel = L.select_learned(csp, w)

    def rec(m):
        x = sel(m)
        if x is not None:
            dec.append(x)
        return x
    c = O.dfs(csp, select=rec)
    d = O.dfs(csp, select=L.select_replay(dec))
    assert (c.nodes, c.fails, c.solutions) == (d.nodes, d.fails, d.solutions) == (b.nodes, b.fails, b.solutions)


def test_mlp_init_layout():
    w = G.mlp_init_weights(3)
    assert w.dtype == np.float32 and w.shape == (L.NW,) and L.NW == 4801
    W1, b1, W2, b2, W3, b3 = L.unpack(w)
    assert np.abs(W1).max() <= math.sqrt(6 / 8) and np.abs(W2).max() <= math.sqrt(6 / 64)
    assert not b1.any() and not b2.any() and b3 == 0
    p = G.epoch_orders(1, 50, 3)
    assert p.shape == (3, 50) and all(sorted(r.tolist()) == list(range(50)) for r in p)
