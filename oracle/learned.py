"""CPU oracle of the learned branching order: TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module; the library never does.

The paper's solver branches first-fail (Sec. 4, search with MiniCP); the learned
order replaces the choice of the branching variable only, so every propagated
domain stays the GAC fixpoint the oracle of ``ct_oracle`` defines. Everything
here is float64 and written from its definition:

Features (NF = 8 per variable; all zero for a variable with |D(x)| < 2). With
s = |D(x)|, d0 its initial size, deg(x) the number of tables whose scope holds x
(degmax the largest deg over the variables, at least 1), smax the largest
domain size among the unfixed variables, and for every table c holding x whose
valid tuples (every component in its current domain) number live_c > 0:
p_c(a) = (valid tuples of c with x = a) / live_c for a in D(x),
    f0 = s / d0                    f4 = mean_c max_a p_c(a)
    f1 = log2(s) / 8               f5 = mean_c (-sum_a p_c(a) log2 p_c(a)) / log2(s)
    f2 = deg(x) / degmax           f6 = mean_c log2(1 + live_c) / 32
    f3 = mean_c s * min_a p_c(a)   f7 = s / smax
(f3-f6 are 0 when no table holding x has a valid tuple; terms with p = 0 add 0).

Network: 3 fully connected layers, 8 -> 64 -> 64 -> 1, ReLU after the first two
(ReLU'(0) = 0). Flat weight vector of 4,801 floats: W1[64][8], b1[64],
W2[64][64], b2[64], W3[64], b3 (rows are output units). Loss of a batch of B
samples: sum_s (out_s - y_s)^2 / (2B). Adam (Kingma and Ba, 2015) with
beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias-corrected moments. Training walks
each epoch's permutation (an input) in consecutive batches, the last one
possibly shorter.

Label of a candidate variable x at a node (the effect of its left branch):
with L = sum_v log2 |D_v| over all variables, propagate D with D(x) := {min D(x)}
to the network's fixpoint; y = 1 if that fails, else (L - L') / L.

Policy: branch on the unfixed variable with the largest score, ties to the
lowest index; left branch x = min D(x), right branch x != min D(x).
"""
from __future__ import annotations

import math

import numpy as np

from oracle import ct_oracle as O

NF = 8
H = 64
NW = H * NF + H + H * H + H + H + 1  # 4801

B1, B2, EPS = 0.9, 0.999, 1e-8


# --------------------------------------------------------------------------
# features
# --------------------------------------------------------------------------

def table_counts(csp: O.Csp, masks):
    """Per table: live_c (number of valid tuples) and, per scope position k, the
    number of valid tuples carrying each value offset of that variable."""
    out = []
    for scope, tup in csp.tables:
        lo = [csp.dom_lo[v] for v in scope]
        sub = [masks[v] for v in scope]
        valid = O.valid_mask(tup, lo, sub)
        vt = tup[valid]
        counts = []
        for k, v in enumerate(scope):
            counts.append(np.bincount(vt[:, k] - csp.dom_lo[v], minlength=csp.dom_size[v]).astype(np.int64))
        out.append((int(valid.sum()), counts))
    return out


def degrees(csp: O.Csp):
    deg = np.zeros(csp.nvars, dtype=np.int64)
    for scope, _ in csp.tables:
        for v in scope:
            deg[v] += 1
    return deg


def features(csp: O.Csp, masks) -> np.ndarray:
    """[nvars, 8] float64 features of every variable (the definition above)."""
    n = csp.nvars
    F = np.zeros((n, NF), dtype=np.float64)
    sizes = np.array([int(m.sum()) for m in masks], dtype=np.int64)
    unfixed = sizes >= 2
    if not unfixed.any():
        return F
    deg = degrees(csp)
    degmax = max(1, int(deg.max()))
    smax = int(sizes[unfixed].max())
    counts = table_counts(csp, masks)
    for x in range(n):
        if not unfixed[x]:
            continue
        s = int(sizes[x])
        vals = np.flatnonzero(masks[x])
        bal, top, ent, liv = [], [], [], []
        for (scope, _), (live, cnt) in zip(csp.tables, counts):
            if x not in scope or live == 0:
                continue
            p = cnt[scope.index(x)][vals].astype(np.float64) / live
            bal.append(s * p.min())
            top.append(p.max())
            nzp = p[p > 0]
            ent.append(-(nzp * np.log2(nzp)).sum() / math.log2(s))
            liv.append(math.log2(1 + live) / 32.0)
        F[x, 0] = s / csp.dom_size[x]
        F[x, 1] = math.log2(s) / 8.0
        F[x, 2] = deg[x] / degmax
        if bal:
            F[x, 3] = float(np.mean(bal))
            F[x, 4] = float(np.mean(top))
            F[x, 5] = float(np.mean(ent))
            F[x, 6] = float(np.mean(liv))
        F[x, 7] = s / smax
    return F


# --------------------------------------------------------------------------
# the network
# --------------------------------------------------------------------------

def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    o = 0
    W1 = w[o:o + H * NF].reshape(H, NF); o += H * NF
    b1 = w[o:o + H]; o += H
    W2 = w[o:o + H * H].reshape(H, H); o += H * H
    b2 = w[o:o + H]; o += H
    W3 = w[o:o + H]; o += H
    b3 = w[o]
    return W1, b1, W2, b2, W3, b3


def forward(w, X) -> np.ndarray:
    """Scores of the rows of X ([n, 8])."""
    W1, b1, W2, b2, W3, b3 = unpack(w)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ W3 + b3


def loss_grad(w, X, y):
    """Loss sum (out - y)^2 / (2B) of the batch and its gradient (flat, like w),
    by the chain rule layer by layer."""
    W1, b1, W2, b2, W3, b3 = unpack(w)
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    B = X.shape[0]
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    out = h2 @ W3 + b3
    r = out - y
    loss = float((r * r).sum() / (2 * B))
    dout = r / B                                  # dL/dout
    gW3 = h2.T @ dout
    gb3 = dout.sum()
    d2 = np.outer(dout, W3) * (z2 > 0)            # dL/dz2
    gW2 = d2.T @ h1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (z1 > 0)                     # dL/dz1
    gW1 = d1.T @ X
    gb1 = d1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
    return loss, g


def adam_step(w, g, m, v, t, lr):
    """One Adam update (t >= 1 is the step count after this update)."""
    m = B1 * m + (1 - B1) * g
    v = B2 * v + (1 - B2) * g * g
    mh = m / (1 - B1 ** t)
    vh = v / (1 - B2 ** t)
    w = w - lr * mh / (np.sqrt(vh) + EPS)
    return w, m, v


def train(w, X, y, perms, batch, lr):
    """Adam over the epochs given by `perms` (one permutation of the samples per
    epoch), consecutive batches of `batch` samples. Returns the weights and the
    mean batch loss of every epoch."""
    w = np.asarray(w, dtype=np.float64).copy()
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    t = 0
    losses = []
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    for perm in perms:
        ls = []
        for s in range(0, len(perm), batch):
            idx = np.asarray(perm[s:s + batch])
            loss, g = loss_grad(w, X[idx], y[idx])
            t += 1
            w, m, v = adam_step(w, g, m, v, t, lr)
            ls.append(loss)
        losses.append(float(np.mean(ls)))
    return w, losses


# --------------------------------------------------------------------------
# labels and the learned search
# --------------------------------------------------------------------------

def log_size(masks) -> float:
    return float(sum(math.log2(int(m.sum())) for m in masks))


def lookahead_label(csp: O.Csp, masks, x: int) -> float:
    """y of candidate x at a node with domains `masks` (a fixpoint)."""
    L = log_size(masks)
    probe = [m.copy() for m in masks]
    a = int(np.flatnonzero(probe[x])[0])
    probe[x][:] = False
    probe[x][a] = True
    st, out, _ = O.gac_network(csp, probe)
    if st == O.INFEASIBLE:
        return 1.0
    return (L - log_size(out)) / L


def select_learned(csp: O.Csp, w):
    """The policy as a select function for ct_oracle.dfs."""
    def select(masks):
        sizes = [int(m.sum()) for m in masks]
        cand = [v for v, s in enumerate(sizes) if s > 1]
        if not cand:
            return None
        sc = forward(w, features(csp, masks))
        best = cand[0]
        for v in cand[1:]:
            if sc[v] > sc[best]:
                best = v
        return best
    return select


def select_replay(decisions):
    """A select function that returns the given branching variables in order
    (depth-first order of the branching nodes); None where all are fixed."""
    it = iter(list(decisions))

    def select(masks):
        if all(int(m.sum()) <= 1 for m in masks):
            return None
        return next(it)
    return select
