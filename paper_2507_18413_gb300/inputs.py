"""Seeded synthetic inputs for table constraints (shared by tests, bench and smoke).

This module holds random-number generation and the shapes of the synthetic
workloads only: tuple lists, scopes and domain-reduction edits. It contains no
part of the propagation arithmetic (no supports, no currTable, no filtering),
so both the CPU oracle and the CUDA path can be fed from it without sharing
any of the method's code.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used in its counter form:
output i of stream ``seed`` is ``mix(seed + i * 0x9E3779B97F4A7C15)``.

The workloads stand in for the paper's instance sets (Sec. 5.1: LIN_B, LIN_EB,
the Gecode set and Orienteering), whose files are not available; their shapes
(arity, domain sizes, tuple counts) follow the synthetic configurations listed
in the project's design notes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, start: int, n: int) -> np.ndarray:
    """Outputs ``start+1 .. start+n`` of the SplitMix64 stream ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class Rng:
    """Sequential view of one SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        self.pos = 0

    def u64(self, n: int) -> np.ndarray:
        out = splitmix64(self.seed, self.pos, n)
        self.pos += n
        return out

    def below(self, n: int, hi) -> np.ndarray:
        """n integers uniform in [0, hi) (hi may be an array); modulo bias < 2^-40 for hi < 2^24."""
        hi = np.asarray(hi, dtype=np.uint64)
        return (self.u64(n) % hi).astype(np.int64)

    def uniform(self, n: int) -> np.ndarray:
        """n doubles uniform in [0, 1) from the top 53 bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def int(self, hi: int) -> int:
        return int(self.below(1, hi)[0])

    def choice(self, seq):
        return seq[self.int(len(seq))]


def derive_seed(*parts: int) -> int:
    """A child seed from a tuple of integers (first output of a stream keyed by them)."""
    s = 0x5EED
    for p in parts:
        s = int(splitmix64((s ^ (int(p) & 0xFFFFFFFFFFFFFFFF)), 0, 1)[0])
    return s


# --------------------------------------------------------------------------
# tuple lists
# --------------------------------------------------------------------------

def _decode(codes: np.ndarray, dom_lo, dom_size) -> np.ndarray:
    """Mixed-radix decode of tuple codes into int32 columns (column 0 least significant)."""
    arity = len(dom_size)
    out = np.empty((codes.shape[0], arity), dtype=np.int32)
    c = codes.copy()
    for i in range(arity):
        d = np.uint64(dom_size[i])
        out[:, i] = (c % d).astype(np.int64) + int(dom_lo[i])
        c //= d
    return out


def distinct_uniform_tuples(seed: int, dom_lo, dom_size, t: int) -> np.ndarray:
    """``t`` distinct tuples drawn uniformly from the product of the domains, in draw order.

    Raises if ``t`` exceeds the number of distinct tuples; callers that may ask for
    more (tiny domains) cap ``t`` first with :func:`cap_distinct`.
    """
    space = 1
    for d in dom_size:
        space *= int(d)
    if t > space:
        raise ValueError(f"cannot draw {t} distinct tuples from a space of {space}")
    if space >= 2 ** 63:
        raise ValueError("tuple space too large for 64-bit codes")
    rng = Rng(seed)
    got = np.empty(0, dtype=np.uint64)
    order = np.empty(0, dtype=np.int64)
    drawn = 0
    while got.shape[0] < t:
        need = t - got.shape[0]
        batch = int(need * 1.25) + 64
        codes = rng.u64(batch) % np.uint64(space)
        allc = np.concatenate([got, codes])
        allo = np.concatenate([order, np.arange(drawn, drawn + batch, dtype=np.int64)])
        drawn += batch
        _, first = np.unique(allc, return_index=True)
        first.sort()
        got = allc[first][:t]
        order = allo[first][:t]
    return _decode(got, dom_lo, dom_size)


def cap_distinct(dom_size, t: int) -> int:
    """Tuple count capped at half the product of the domain sizes (distinct draws must end)."""
    space = math.prod(int(d) for d in dom_size)
    return int(min(t, max(1, space // 2)))


def zipf_tuples(seed: int, dom_lo, dom_size, t: int, s: float = 1.2) -> np.ndarray:
    """``t`` tuples (duplicates allowed) whose columns are independent Zipf(s) draws.

    Value rank k (0-based) of column i has probability proportional to (k+1)^-s; the
    rank is mapped to the value ``dom_lo[i] + perm_i[k]`` with a seeded permutation so
    that the heavy values are not always the smallest ones.
    """
    rng = Rng(seed)
    arity = len(dom_size)
    out = np.empty((t, arity), dtype=np.int32)
    for i in range(arity):
        d = int(dom_size[i])
        w = 1.0 / np.power(np.arange(1, d + 1, dtype=np.float64), s)
        cdf = np.cumsum(w)
        cdf /= cdf[-1]
        u = rng.uniform(t)
        rank = np.minimum(np.searchsorted(cdf, u, side="right"), d - 1)
        perm = np.argsort(rng.u64(d), kind="stable")
        out[:, i] = perm[rank].astype(np.int64) + int(dom_lo[i])
    return out


def random_scope(rng: Rng, nvars: int, arity: int) -> list:
    """``arity`` distinct variable indices in [0, nvars), in draw order."""
    picked = []
    while len(picked) < arity:
        v = rng.int(nvars)
        if v not in picked:
            picked.append(v)
    return picked


# --------------------------------------------------------------------------
# domain-reduction streams (what a search would do between propagations)
# --------------------------------------------------------------------------

def present_values(mask: np.ndarray) -> np.ndarray:
    return np.flatnonzero(mask)


def remove_random_values(rng: Rng, masks: list, k: int, min_left: int = 1):
    """Remove up to ``k`` present values, each from a random variable with more than
    ``min_left`` values left. Returns the new masks (copies) and the number removed."""
    masks = [m.copy() for m in masks]
    removed = 0
    for _ in range(k):
        cand = [i for i, m in enumerate(masks) if int(m.sum()) > min_left]
        if not cand:
            break
        i = cand[rng.int(len(cand))]
        vals = present_values(masks[i])
        a = int(vals[rng.int(len(vals))])
        masks[i][a] = False
        removed += 1
    return masks, removed


def delta_step(rng: Rng, masks: list):
    """Remove 1-2 values of one variable that has at least 3 values (a delta-path edit)."""
    masks = [m.copy() for m in masks]
    cand = [i for i, m in enumerate(masks) if int(m.sum()) >= 3]
    if not cand:
        return masks, None
    i = cand[rng.int(len(cand))]
    vals = present_values(masks[i])
    k = 1 + rng.int(2)
    k = min(k, len(vals) - 1)
    pick = rng.below(len(vals), 1 << 62)
    order = np.argsort(pick, kind="stable")[:k]
    masks[i][vals[order]] = False
    return masks, i


def reset_step(rng: Rng, masks: list):
    """Remove more than half of one variable's values, leaving at least one (a reset-path edit).

    The count removed is uniform in [ceil(|D|/2)+1, |D|-1] for a variable with |D| >= 4.
    """
    masks = [m.copy() for m in masks]
    cand = [i for i, m in enumerate(masks) if int(m.sum()) >= 4]
    if not cand:
        return masks, None
    i = cand[rng.int(len(cand))]
    vals = present_values(masks[i])
    n = len(vals)
    lo = (n + 1) // 2 + 1
    hi = n - 1
    k = lo + rng.int(hi - lo + 1)
    pick = rng.below(n, 1 << 62)
    order = np.argsort(pick, kind="stable")[:k]
    masks[i][vals[order]] = False
    return masks, i


# --------------------------------------------------------------------------
# workload descriptions
# --------------------------------------------------------------------------

@dataclass
class TableSpec:
    scope: list
    tuples: np.ndarray  # int32 [t, arity], actual values


@dataclass
class CspSpec:
    nvars: int
    dom_lo: list
    dom_size: list
    tables: list = field(default_factory=list)


def tiny_table(seed: int = 1):
    """Arity 3, domains {0..7}, 200 distinct uniform tuples."""
    dom_lo, dom_size = [0, 0, 0], [8, 8, 8]
    return dom_lo, dom_size, distinct_uniform_tuples(seed, dom_lo, dom_size, 200)


def large_table(seed: int, t: int, arity: int = 6, d: int = 32):
    """Arity 6, 32-value domains {0..31}, ``t`` distinct uniform tuples."""
    dom_lo, dom_size = [0] * arity, [d] * arity
    return dom_lo, dom_size, distinct_uniform_tuples(seed, dom_lo, dom_size, t)


def random_csp(seed: int, nvars: int, ntables: int, arity: int, d: int, t: int,
               dist: str = "uniform") -> CspSpec:
    """``ntables`` tables of ``arity`` over random distinct-within-table scopes of ``nvars``
    variables with domains {0..d-1}; ``t`` tuples each (distinct uniform or Zipf)."""
    rng = Rng(seed)
    csp = CspSpec(nvars=nvars, dom_lo=[0] * nvars, dom_size=[d] * nvars)
    for k in range(ntables):
        scope = random_scope(rng, nvars, arity)
        ts = derive_seed(seed, k)
        if dist == "uniform":
            tt = cap_distinct([d] * arity, t)
            tup = distinct_uniform_tuples(ts, [0] * arity, [d] * arity, tt)
        else:
            tup = zipf_tuples(ts, [0] * arity, [d] * arity, t)
        csp.tables.append(TableSpec(scope=scope, tuples=tup))
    return csp


def batching_csp(seed: int, nvars: int = 40, ntables: int = 60, arity: int = 4, d: int = 24,
                 t_lo: float = 1e4, t_hi: float = 2e5) -> CspSpec:
    """The search workload of the batching experiments: ``ntables`` tables of ``arity``
    over random scopes of ``nvars`` variables with domains {0..d-1}, each holding a
    log-uniform number of distinct uniform tuples in [t_lo, t_hi] (capped at half the
    tuple space). With the defaults the expected solution count is of order one (the
    product of the table densities times d^nvars), i.e. near the satisfiability threshold."""
    rng = Rng(seed)
    csp = CspSpec(nvars=nvars, dom_lo=[0] * nvars, dom_size=[d] * nvars)
    for k in range(ntables):
        scope = random_scope(rng, nvars, arity)
        u = float(rng.uniform(1)[0])
        t = int(round(math.exp(math.log(t_lo) + u * (math.log(t_hi) - math.log(t_lo)))))
        t = cap_distinct([d] * arity, t)
        tup = distinct_uniform_tuples(derive_seed(seed, k), [0] * arity, [d] * arity, t)
        csp.tables.append(TableSpec(scope=scope, tuples=tup))
    return csp


# --------------------------------------------------------------------------
# learned branching order: initial weights, epoch orders, instances
# --------------------------------------------------------------------------

MLP_NF, MLP_H = 8, 64
MLP_NW = MLP_H * MLP_NF + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1


def mlp_init_weights(seed: int) -> np.ndarray:
    """Initial float32 weights of the 8 -> 64 -> 64 -> 1 network, flat in the order
    W1[64][8], b1, W2[64][64], b2, W3[64], b3: weights uniform in +-sqrt(6 / fan_in)
    (He et al., 2015, uniform form), biases zero."""
    rng = Rng(seed)
    w = np.zeros(MLP_NW, dtype=np.float64)
    o = 0
    for fan_in, n in ((MLP_NF, MLP_H * MLP_NF), (None, MLP_H), (MLP_H, MLP_H * MLP_H), (None, MLP_H),
                      (MLP_H, MLP_H), (None, 1)):
        if fan_in is not None:
            a = math.sqrt(6.0 / fan_in)
            w[o:o + n] = (rng.uniform(n) * 2.0 - 1.0) * a
        o += n
    return w.astype(np.float32)


def epoch_orders(seed: int, n: int, epochs: int) -> np.ndarray:
    """[epochs, n] int32: one seeded permutation of the n training samples per epoch."""
    rng = Rng(seed)
    return np.stack([np.argsort(rng.u64(n), kind="stable").astype(np.int32) for _ in range(epochs)])


def learned_csp(seed: int, nvars=(30, 60), dom=(16, 64), ntables=(40, 120), arity=(3, 6),
                tuples=(1e4, 5e5), log2_solutions: float = 4.0) -> CspSpec:
    """A random CSP for the learned-order experiments: the number of variables,
    each domain size, the number of tables and each arity uniform in the given
    inclusive ranges; random scopes. Each table's tuple count is its share of a
    target expected solution count of 2^log2_solutions (the product of the
    table densities times the product of the domain sizes), clamped to the
    `tuples` range and to half the tuple space; distinct uniform tuples."""
    rng = Rng(seed)
    nv = nvars[0] + rng.int(nvars[1] - nvars[0] + 1)
    sizes = [dom[0] + rng.int(dom[1] - dom[0] + 1) for _ in range(nv)]
    nt = ntables[0] + rng.int(ntables[1] - ntables[0] + 1)
    scopes = [random_scope(rng, nv, arity[0] + rng.int(arity[1] - arity[0] + 1)) for _ in range(nt)]
    space_bits = sum(math.log2(d) for d in sizes)
    # log2 density per table so that space_bits + sum(log2 density) = log2_solutions
    per_table = (log2_solutions - space_bits) / nt
    csp = CspSpec(nvars=nv, dom_lo=[0] * nv, dom_size=sizes)
    for k, sc in enumerate(scopes):
        ds = [sizes[v] for v in sc]
        tbits = sum(math.log2(d) for d in ds)
        t = int(round(2.0 ** (tbits + per_table)))
        t = max(int(tuples[0]), min(int(tuples[1]), t))
        t = cap_distinct(ds, t)
        tup = distinct_uniform_tuples(derive_seed(seed, k), [0] * len(sc), ds, t)
        csp.tables.append(TableSpec(scope=sc, tuples=tup))
    return csp


STAR = -2 ** 31  # the wildcard component of a short tuple


def short_tuples(seed: int, dom_lo, dom_size, t: int, star_prob: float = 0.2) -> np.ndarray:
    """``t`` distinct uniform tuples in which every component is independently
    replaced by the wildcard STAR with probability ``star_prob`` (seeded)."""
    tup = distinct_uniform_tuples(seed, dom_lo, dom_size, t).astype(np.int64)
    rng = Rng(derive_seed(seed, 0x5747))
    u = rng.uniform(tup.size).reshape(tup.shape)
    tup[u < star_prob] = STAR
    return tup.astype(np.int32)


def network_tables(seed: int, ntables: int = 512, nvars: int = 1024, arity=(2, 8), tuples=(1e3, 1e6),
                   dom=(8, 128), zipf_s: float = 1.2) -> CspSpec:
    """The many-table network of the batching experiments: ``nvars`` variables with
    domain sizes uniform in ``dom``; ``ntables`` tables of arity uniform in ``arity``
    over random scopes, each with a log-uniform tuple count in ``tuples``. Even
    tables hold distinct uniform tuples (capped at half the tuple space), odd
    tables per-column Zipf(zipf_s) tuples (duplicates possible)."""
    rng = Rng(seed)
    sizes = [dom[0] + rng.int(dom[1] - dom[0] + 1) for _ in range(nvars)]
    csp = CspSpec(nvars=nvars, dom_lo=[0] * nvars, dom_size=sizes)
    lo, hi = math.log(tuples[0]), math.log(tuples[1])
    for k in range(ntables):
        a = arity[0] + rng.int(arity[1] - arity[0] + 1)
        sc = random_scope(rng, nvars, a)
        ds = [sizes[v] for v in sc]
        t = int(round(math.exp(lo + float(rng.uniform(1)[0]) * (hi - lo))))
        ts = derive_seed(seed, k)
        if k % 2 == 0:
            tup = distinct_uniform_tuples(ts, [0] * a, ds, cap_distinct(ds, t))
        else:
            tup = zipf_tuples(ts, [0] * a, ds, t, s=zipf_s)
        csp.tables.append(TableSpec(scope=sc, tuples=tup))
    return csp


def planning_csp(seed: int, states: int = 256, actions: int = 32, horizon: int = 30, alternatives=(0, 3)) -> CspSpec:
    """A planning-style chain: state variables s_0..s_H (domain 0..states-1) and
    action variables a_0..a_{H-1} (0..actions-1), one transition table
    T(s_t, a_t, s_{t+1}) per step holding, for every (s, a), its successor plus
    0-3 alternatives drawn uniformly (the same relation at every step). s_0 is
    fixed to state 0 and s_H to the end of a seeded random walk of H steps from
    it, so at least one plan exists. Variables: s_t is t, a_t is H + 1 + t."""
    rng = Rng(seed)
    succ = rng.below(states * actions, states).reshape(states, actions)
    rows = []
    for st in range(states):
        for ac in range(actions):
            nxt = [int(succ[st, ac])]
            k = alternatives[0] + rng.int(alternatives[1] - alternatives[0] + 1)
            while len(nxt) < 1 + k:
                c = rng.int(states)
                if c not in nxt:
                    nxt.append(c)
            rows.extend((st, ac, n) for n in nxt)
    tup = np.asarray(rows, dtype=np.int32)
    cur = 0
    for _ in range(horizon):
        cur = int(succ[cur, rng.int(actions)])
    nv = 2 * horizon + 1
    lo = [0] * nv
    size = [states] * (horizon + 1) + [actions] * horizon
    lo[0], size[0] = 0, 1
    lo[horizon], size[horizon] = cur, 1
    csp = CspSpec(nvars=nv, dom_lo=lo, dom_size=size)
    for t in range(horizon):
        csp.tables.append(TableSpec(scope=[t, horizon + 1 + t, t + 1], tuples=tup))
    return csp

