"""GPU parity of the learned branching order against its float64 oracle
(oracle/learned.py): features, network inference, gradients and training to
1e-4 relative, lookahead labels, and searches whose decisions the oracle
replays (each decision the oracle's best score within the float32 tolerance)."""
import math

import numpy as np
import pytest

from oracle import ct_oracle as O
from oracle import learned as L
from paper_2507_18413_gb300 import ct as C
from paper_2507_18413_gb300 import inputs as G
from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


def _model(csp, raw, host_fixpoint=0):
    torch = torch_cuda()
    C.load()
    st, h = C.ct_model_create(csp.dom_lo, csp.dom_size, opt=C.make_options(host_fixpoint=host_fixpoint),
                              stream=torch.cuda.current_stream())
    assert st == C.CT_OK, C.last_error()
    for scope, tup in raw:
        assert C.ct_model_add_table(h, scope, tup) >= 0, C.last_error()
    return h


def _random(seed, nvars, ntables, arity, dlo, dhi, t):
    rng = G.Rng(seed)
    sizes = [dlo + rng.int(dhi - dlo + 1) for _ in range(nvars)]
    csp = O.Csp([0] * nvars, sizes)
    raw = []
    for k in range(ntables):
        sc = G.random_scope(rng, nvars, arity)
        ds = [sizes[v] for v in sc]
        tup = G.distinct_uniform_tuples(G.derive_seed(seed, k), [0] * arity, ds, G.cap_distinct(ds, t))
        csp.add_table(sc, tup)
        raw.append((sc, tup))
    return csp, raw


def _weights(seed):
    """Initial weights plus non-zero biases, so that both ReLU sides occur."""
    w = G.mlp_init_weights(seed).astype(np.float64)
    rng = G.Rng(seed + 1000)
    b1 = slice(L.H * L.NF, L.H * L.NF + L.H)
    b2 = slice(L.H * L.NF + L.H + L.H * L.H, L.H * L.NF + L.H + L.H * L.H + L.H)
    w[b1] = (rng.uniform(L.H) - 0.5) * 0.4
    w[b2] = (rng.uniform(L.H) - 0.5) * 0.4
    w[-1] = 0.1
    return w.astype(np.float32)


def _masks(h, csp):
    off, _ = C.dom_layout(csp.dom_size)
    st, w = C.ct_model_get_domains(h, int(off[-1]))
    assert st == C.CT_OK
    return C.words_to_masks(w, csp.dom_size)


@pytest.mark.parametrize("seed", range(4))
def test_features_match_the_oracle(seed):
    # multi-word domains (d up to 40) and tables of several segments (up to 12,000 tuples)
    csp, raw = _random(700 + seed, nvars=9, ntables=6, arity=3, dlo=5, dhi=40, t=12_000)
    h = _model(csp, raw)
    assert C.ct_model_propagate(h) in (C.CT_OK, C.CT_INFEASIBLE)
    rng = G.Rng(seed)
    for step in range(6):
        masks = _masks(h, csp)
        st, F = C.ct_model_features(h, csp.nvars)
        assert st == C.CT_OK, C.last_error()
        want = L.features(csp, masks)
        assert np.allclose(F, want, rtol=1e-5, atol=1e-6), np.abs(F - want).max()
        # shrink a domain and propagate to the next state
        new, _ = G.delta_step(rng, masks)
        assert C.ct_model_set_domains(h, C.masks_to_words(new)) == C.CT_OK
        if C.ct_model_propagate(h) != C.CT_OK:
            break
    C.ct_model_destroy(h)


def test_inference_matches_the_oracle():
    torch = torch_cuda()
    C.load()
    w = _weights(3)
    st, net = C.ct_mlp_create(w, stream=torch.cuda.current_stream())
    assert st == C.CT_OK, C.last_error()
    rng = np.random.default_rng(4)
    for n in (1, 37, 1000, 4099):
        X = rng.random((n, 8)).astype(np.float32) * 1.5 - 0.25
        xd = torch.from_numpy(X).cuda()
        sd = torch.zeros(n, dtype=torch.float32, device="cuda")
        assert C.ct_mlp_forward(net, xd, n, sd) == C.CT_OK
        got = sd.cpu().numpy().astype(np.float64)
        want = L.forward(w.astype(np.float64), X.astype(np.float64))
        assert np.all(np.abs(got - want) <= 1e-4 * np.maximum(1.0, np.abs(want))), np.abs(got - want).max()
    C.ct_mlp_destroy(net)


@pytest.mark.parametrize("n", [1, 50, 128])
def test_gradient_matches_the_oracle(n):
    torch = torch_cuda()
    C.load()
    w = _weights(5)
    st, net = C.ct_mlp_create(w, stream=torch.cuda.current_stream())
    assert st == C.CT_OK
    rng = np.random.default_rng(n)
    X = rng.random((n, 8)).astype(np.float32)
    y = rng.random(n).astype(np.float32)
    st, loss, g = C.ct_mlp_grad(net, X, y)
    assert st == C.CT_OK, C.last_error()
    lw, gw = L.loss_grad(w.astype(np.float64), X.astype(np.float64), y.astype(np.float64))
    assert math.isclose(loss, lw, rel_tol=1e-4)
    assert np.linalg.norm(g - gw) <= 1e-4 * np.linalg.norm(gw)
    st, w2 = C.ct_mlp_get_weights(net)
    assert np.array_equal(w2, w), "the gradient call changed the weights"
    C.ct_mlp_destroy(net)


def test_training_matches_the_oracle():
    """Three epochs of Adam over 300 samples in batches of 64 (a short last batch)."""
    torch = torch_cuda()
    C.load()
    w0 = _weights(7)
    st, net = C.ct_mlp_create(w0, stream=torch.cuda.current_stream())
    assert st == C.CT_OK
    rng = np.random.default_rng(8)
    X = rng.random((300, 8)).astype(np.float32)
    y = (0.6 * X[:, 0] - 0.2 * X[:, 5] + 0.1).astype(np.float32)
    orders = G.epoch_orders(3, 300, 3)
    st, losses = C.ct_mlp_train(net, X, y, orders, 64, 1e-3)
    assert st == C.CT_OK, C.last_error()
    st, w = C.ct_mlp_get_weights(net)
    ww, lw = L.train(w0.astype(np.float64), X.astype(np.float64), y.astype(np.float64), orders, 64, 1e-3)
    assert np.allclose(losses, lw, rtol=1e-4)
    assert np.linalg.norm(w - ww) <= 1e-4 * np.linalg.norm(ww)
    # training continues from the kept Adam state
    st, losses2 = C.ct_mlp_train(net, X, y, G.epoch_orders(4, 300, 2), 64, 1e-3)
    assert st == C.CT_OK and losses2[-1] < losses[0]
    C.ct_mlp_destroy(net)


@pytest.mark.parametrize("seed", range(3))
def test_lookahead_labels_match_the_oracle(seed):
    csp, raw = _random(800 + seed, nvars=8, ntables=6, arity=3, dlo=4, dhi=9, t=150)
    h = _model(csp, raw)
    if C.ct_model_propagate(h) != C.CT_OK:
        pytest.skip("root infeasible")
    masks = _masks(h, csp)
    for slots in (1, 3, 16):
        st, lab = C.ct_model_lookahead(h, csp.nvars, slots)
        assert st == C.CT_OK, C.last_error()
        for v in range(csp.nvars):
            if masks[v].sum() < 2:
                assert math.isnan(lab[v])
            else:
                assert abs(lab[v] - L.lookahead_label(csp, masks, v)) <= 1e-6, (slots, v)
    # the model itself is untouched
    assert all(np.array_equal(a, b) for a, b in zip(_masks(h, csp), masks))
    C.ct_model_destroy(h)


def _checked_replay(csp, w, decisions):
    """Oracle select: replays the library's decisions and checks that each is the
    float64 argmax up to the float32 tolerance."""
    it = iter(decisions)

    def select(masks):
        if all(int(m.sum()) <= 1 for m in masks):
            return None
        x = next(it)
        sc = L.forward(w.astype(np.float64), L.features(csp, masks))
        cand = [v for v, m in enumerate(masks) if m.sum() > 1]
        assert x in cand
        best = max(sc[v] for v in cand)
        assert sc[x] >= best - 1e-4 * max(1.0, abs(best)), (x, sc[x], best)
        return x
    return select


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("seed", range(3))
def test_learned_search_is_replayed_by_the_oracle(seed, mode):
    torch = torch_cuda()
    csp, raw = _random(900 + seed, nvars=8, ntables=5, arity=3, dlo=4, dhi=7, t=60)
    h = _model(csp, raw, host_fixpoint=mode)
    w = _weights(20 + seed)
    st, net = C.ct_mlp_create(w, stream=torch.cuda.current_stream())
    assert st == C.CT_OK
    assert C.ct_model_set_policy(h, net) == C.CT_OK
    tr = C.Trace(100_000)
    assert C.ct_model_set_trace(h, tr) == C.CT_OK
    st, got = C.ct_search_dfs(h, csp.nvars, 0, True)
    assert st == C.CT_OK, C.last_error()
    dec = tr.decisions()
    want = O.dfs(csp, select=_checked_replay(csp, w, dec))
    assert (got["nodes"], got["fails"], got["solutions"]) == (want.nodes, want.fails, want.solutions)
    assert got["max_depth"] == want.max_depth
    if want.solutions:
        assert got["first_solution"] == want.first_solution
    # the batched search with the same policy visits the same tree
    for slots, split in ((8, 2), (32, 0)):
        st, b, _ = C.ct_search_batch(h, csp.nvars, slots, split, 0, True)
        assert st == C.CT_OK, C.last_error()
        for k in ("nodes", "fails", "solutions", "max_depth", "first_solution"):
            assert b[k] == got[k], k
    # first-fail again without the policy
    assert C.ct_model_set_policy(h, None) == C.CT_OK
    st, ff = C.ct_search_dfs(h, csp.nvars, 0, True)
    ref = O.dfs(csp)
    assert (ff["nodes"], ff["solutions"]) == (ref.nodes, ref.solutions)
    C.ct_model_set_trace(h, None)
    C.ct_model_destroy(h)
    C.ct_mlp_destroy(net)


def test_collected_samples_and_training_end_to_end():
    torch = torch_cuda()
    csp, raw = _random(1234, nvars=10, ntables=8, arity=3, dlo=4, dhi=8, t=120)
    h = _model(csp, raw)
    st, X, y = C.ct_search_collect(h, 400, 16, 5000)
    assert st == C.CT_OK, C.last_error()
    assert len(y) > 50
    assert np.all((y >= 0) & (y <= 1)) and np.all(np.isfinite(X))
    assert np.all((X[:, 0] > 0) & (X[:, 0] <= 1)) and np.all(X[:, 7] <= 1)
    # the first sample block is the root's unfixed variables: oracle features and labels
    assert C.ct_model_propagate(h) == C.CT_OK
    masks = _masks(h, csp)
    root = [v for v in range(csp.nvars) if masks[v].sum() > 1]
    Fo = L.features(csp, masks)
    for i, v in enumerate(root):
        assert np.allclose(X[i], Fo[v], rtol=1e-5, atol=1e-6)
        assert abs(y[i] - L.lookahead_label(csp, masks, v)) <= 1e-6
    st, net = C.ct_mlp_create(G.mlp_init_weights(1), stream=torch.cuda.current_stream())
    st, losses = C.ct_mlp_train(net, X, y, G.epoch_orders(2, len(y), 20), 64, 3e-3)
    assert st == C.CT_OK and losses[-1] < losses[0]
    C.ct_mlp_destroy(net)
    C.ct_model_destroy(h)


def test_bad_arguments():
    torch_cuda()
    C.load()
    st, net = C.ct_mlp_create(G.mlp_init_weights(1))
    assert st == C.CT_OK
    X = np.zeros((129, 8), np.float32)
    assert C.ct_mlp_grad(net, X, np.zeros(129, np.float32))[0] == C.CT_ERR_ARG
    bad = np.zeros((1, 10), np.int32)
    bad[0, 3] = 10
    assert C.ct_mlp_train(net, np.zeros((10, 8), np.float32), np.zeros(10, np.float32), bad, 4, 1e-3)[0] == C.CT_ERR_ARG
    C.ct_mlp_destroy(net)
