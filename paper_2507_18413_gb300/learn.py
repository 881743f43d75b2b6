"""Training and evaluation driver of the learned branching order (host side).

Every step of the arithmetic runs in the library's kernels (features, lookahead
propagations, the network, Adam); this module only sequences the C ABI calls:
build a model per instance, collect (features, label) samples along plain
first-fail searches, train the network, and compare searches with and without
it on held-out instances.
"""
from __future__ import annotations

import time

import numpy as np

from . import ct as C
from . import inputs as G


def build_model(spec, stream=None):
    """A ct_model holding the instance (inputs.CspSpec)."""
    st, m = C.ct_model_create(spec.dom_lo, spec.dom_size, stream=stream)
    C.check(st)
    for tb in spec.tables:
        st = C.ct_model_add_table(m, tb.scope, tb.tuples)
        if st < 0:
            C.check(st)
    return m


def collect(specs, node_limit=2000, slots=64, max_samples=100_000, stream=None):
    """Samples from first-fail searches of the instances, up to max_samples in all."""
    Xs, ys = [], []
    n = 0
    for spec in specs:
        if n >= max_samples:
            break
        m = build_model(spec, stream)
        try:
            st, X, y = C.ct_search_collect(m, node_limit, slots, max_samples - n)
            C.check(st)
        finally:
            C.ct_model_destroy(m)
        Xs.append(X)
        ys.append(y)
        n += len(y)
    if not Xs:
        return np.zeros((0, C.MLP_FEATURES), np.float32), np.zeros(0, np.float32)
    return np.concatenate(Xs), np.concatenate(ys)


def train(X, y, seed=1, epochs=20, batch=128, lr=1e-3, stream=None):
    """A network trained on the samples; returns (handle, epoch losses)."""
    st, net = C.ct_mlp_create(G.mlp_init_weights(seed), stream=stream)
    C.check(st)
    st, losses = C.ct_mlp_train(net, X, y, G.epoch_orders(seed + 1, len(y), epochs), batch, lr)
    C.check(st)
    return net, losses


def solve(spec, policy=None, batched=None, node_limit=100_000, stream=None):
    """Search for the first solution (or a proof of infeasibility) with first-fail
    (policy None) or the network; batched = (slots, split_depth) for the batched
    search. Returns the search counters."""
    m = build_model(spec, stream)
    try:
        if policy is not None:
            C.check(C.ct_model_set_policy(m, policy))
        if batched:
            # the batched search stops at the first solution any slot finds
            st, d, info = C.ct_search_batch(m, spec.nvars, batched[0], batched[1], node_limit, "any")
        else:
            st, d = C.ct_search_dfs(m, spec.nvars, node_limit, False)
        C.check(st)
    finally:
        C.ct_model_destroy(m)
    return d


ARMS = ("first_fail", "learned", "first_fail_batched", "learned_batched")


def compare(specs, policy, node_limit=100_000, batched=(64, 6), stream=None):
    """First-fail against the network, plain and batched, on the instances: per
    instance and arm the nodes, seconds and whether the search finished (a
    solution or a proof of infeasibility) within the node limit."""
    rows = []
    for spec in specs:
        row = {"nvars": spec.nvars, "tables": len(spec.tables)}
        row["first_fail"] = _brief(solve(spec, None, None, node_limit, stream))
        row["learned"] = _brief(solve(spec, policy, None, node_limit, stream))
        if batched:
            row["first_fail_batched"] = _brief(solve(spec, None, batched, node_limit, stream))
            row["learned_batched"] = _brief(solve(spec, policy, batched, node_limit, stream))
        rows.append(row)
    return rows


def summarize(rows):
    """Per arm: instances finished, total nodes and seconds, and the geometric
    means over the instances every arm finished of nodes and seconds relative
    to plain first-fail."""
    import math
    arms = [a for a in ARMS if rows and a in rows[0]]
    both = [r for r in rows if all(r[a]["finished"] for a in arms)]
    out = {"instances": len(rows), "finished_by_all": len(both)}
    for a in arms:
        d = {"finished": sum(1 for r in rows if r[a]["finished"]),
             "nodes": int(sum(r[a]["nodes"] for r in rows)),
             "seconds": round(sum(r[a]["seconds"] for r in rows), 3)}
        if both:
            d["geomean_nodes_vs_first_fail"] = round(math.exp(sum(
                math.log(max(1, r[a]["nodes"]) / max(1, r["first_fail"]["nodes"])) for r in both) / len(both)), 3)
            d["geomean_time_vs_first_fail"] = round(math.exp(sum(
                math.log(max(1e-6, r[a]["seconds"]) / max(1e-6, r["first_fail"]["seconds"])) for r in both)
                / len(both)), 3)
        out[a] = d
    return out


def _brief(d):
    return {"nodes": d["nodes"], "seconds": round(d["seconds"], 4), "finished": bool(d["complete"]),
            "solution": d["solutions"] > 0}
