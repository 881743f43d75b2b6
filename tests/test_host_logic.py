"""Host-side logic that runs without a GPU: the seeded workload generators'
structure, the learned-order comparison summary, and the all-cores CPU
baseline of the bench."""
import math
import types

import numpy as np
import pytest

from oracle import ct_oracle as O
from paper_2507_18413_gb300 import ct as C
from paper_2507_18413_gb300 import inputs as G
from paper_2507_18413_gb300 import learn as L


def test_planning_chain_structure_and_a_plan_exists():
    """Variables s_0..s_H then a_0..a_{H-1}; s_0 and s_H fixed; every step's
    table holds each (s, a)'s successor plus 0-3 alternatives, the same
    relation at every step; the oracle's search finds a plan."""
    H, S, A = 5, 12, 3
    spec = G.planning_csp(4, states=S, actions=A, horizon=H)
    assert spec.nvars == 2 * H + 1
    assert spec.dom_size[0] == 1 and spec.dom_lo[0] == 0 and spec.dom_size[H] == 1
    assert spec.dom_size[1:H] == [S] * (H - 1) and spec.dom_size[H + 1:] == [A] * H
    rel = spec.tables[0].tuples
    for t, tb in enumerate(spec.tables):
        assert tb.scope == [t, H + 1 + t, t + 1]
        assert np.array_equal(tb.tuples, rel)
    pairs, counts = np.unique(rel[:, :2], axis=0, return_counts=True)
    assert len(pairs) == S * A and counts.min() >= 1 and counts.max() <= 4
    assert len(np.unique(rel, axis=0)) == len(rel), "successor and alternatives are distinct"
    csp = O.Csp(spec.dom_lo, spec.dom_size)
    for tb in spec.tables:
        csp.add_table(tb.scope, tb.tuples)
    r = O.dfs(csp, count_all=False)
    assert r.solutions == 1 and r.first_solution[0] == 0


def test_network_tables_shapes():
    spec = G.network_tables(7, ntables=24, nvars=40, arity=(2, 5), tuples=(50, 400), dom=(4, 9))
    assert len(spec.tables) == 24 and spec.nvars == 40
    assert all(4 <= d <= 9 for d in spec.dom_size)
    for k, tb in enumerate(spec.tables):
        a = len(tb.scope)
        assert 2 <= a <= 5 and len(set(tb.scope)) == a
        ds = np.array([spec.dom_size[v] for v in tb.scope])
        assert tb.tuples.shape[1] == a
        assert (tb.tuples >= 0).all() and (tb.tuples < ds).all()
        if k % 2 == 0:  # distinct uniform tuples
            assert len(np.unique(tb.tuples, axis=0)) == len(tb.tuples)
    again = G.network_tables(7, ntables=24, nvars=40, arity=(2, 5), tuples=(50, 400), dom=(4, 9))
    assert all(np.array_equal(a.tuples, b.tuples) for a, b in zip(spec.tables, again.tables)), "seeded"


def _row(ff, lr, ffb=None, lrb=None):
    def arm(n, s, fin=True):
        return {"nodes": n, "seconds": s, "finished": fin, "solution": True}
    r = {"nvars": 5, "tables": 3, "first_fail": arm(*ff), "learned": arm(*lr)}
    if ffb:
        r["first_fail_batched"] = arm(*ffb)
        r["learned_batched"] = arm(*lrb)
    return r


def test_learned_summary_arithmetic():
    rows = [_row((100, 1.0), (50, 2.0), (80, 0.5), (40, 0.25)),
            _row((10, 0.1), (40, 0.4), (10, 0.2), (5, 0.05)),
            _row((30, 0.3, False), (20, 0.2), (30, 0.3), (20, 0.2))]
    s = L.summarize(rows)
    assert s["instances"] == 3 and s["finished_by_all"] == 2
    assert s["first_fail"]["finished"] == 2 and s["learned"]["finished"] == 3
    assert s["learned"]["nodes"] == 110 and math.isclose(s["learned"]["seconds"], 2.6)
    # geometric means over the two instances every arm finished
    assert math.isclose(s["learned"]["geomean_nodes_vs_first_fail"], round(math.sqrt(0.5 * 4.0), 3))
    assert math.isclose(s["learned"]["geomean_time_vs_first_fail"], round(math.sqrt(2.0 * 4.0), 3))
    assert math.isclose(s["learned_batched"]["geomean_nodes_vs_first_fail"], round(math.sqrt(0.4 * 0.5), 3))
    assert s["first_fail"]["geomean_nodes_vs_first_fail"] == 1.0


def test_all_cores_cpu_baseline_replays_the_plans():
    """One replica per core replays save / propagate / restore plans of a
    small table and reports propagations per second over its threads."""
    bench = pytest.importorskip("bench")
    dom_lo, dom_size, tup = G.large_table(seed=1, t=3000, arity=4, d=8)
    rng = G.Rng(3)
    plans = []
    for s in range(3):
        rp = types.SimpleNamespace(inputs=[], ops=[])
        masks = [np.ones(d, bool) for d in dom_size]
        for c in range(4):
            new = bench.next_edit(rng, masks)
            rp.inputs.append(C.masks_to_words(new))
            rp.ops += [("save",), ("prop", c)]
            masks = new
        rp.ops.append(("restore", 1))
        plans.append(rp)
    r = bench.cpu_bitset_baseline_cores(types.SimpleNamespace(), plans, dom_lo, dom_size, tup, seconds=0.3)
    assert r["cores"] >= 1 and r["value"] > 0
    assert r["kind"].startswith("serial bitset CT")


class _FakeSampler:
    """Stands in for the nvidia-smi process of the bench's clock record."""

    def __init__(self, text):
        self.text = text

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.text, ""


def test_clock_record_parsing():
    bench = pytest.importorskip("bench")
    lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 2055, 2070, 1390.2, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 1980, 2070, 1400.0, 0x8, Active, Not Active, Not Active, Active",
             "garbage line"]
    r = bench.clocks_stop(_FakeSampler("\n".join(lines) + "\n"))
    assert r["samples"] == 3 and r["sm_mhz"] == 2055.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.clocks_stop(_FakeSampler("")) is None
    assert bench.clocks_stop(None) is None


def test_bench_summary_of_a_line():
    """The line's closing summary: the headline figures, and the other
    configurations' when the line holds them."""
    bench = pytest.importorskip("bench")
    r = {"value": 40000.0, "e2e": {"value": 38000.04}, "roofline": {"frac": 0.017},
         "call_latency_us": {"p50": 21.0}, "cpu_baseline_bitset": {"value": 900.0}}
    s = bench.summary(r)
    assert s["props_per_s"] == 40000.0 and s["e2e_props_per_s"] == 38000.0 and s["roofline_frac"] == 0.017
    assert s["cpu_bitset_1_core"] == 900.0 and s["cpu_bitset_all_cores"] is None and "error" not in s
    r["bulk_update"] = {"t1e6_arity6_d32": {"frac_of_hbm": 0.1, "update_phase_frac_of_hbm": 0.2,
                                            "frac_of_read_ceiling": 0.5}}
    r["stream_1e7_arity5_d64"] = {"value": 29000.0, "roofline": {"frac": 0.04}}
    r["early_filter_ablation"] = {"default_props_per_s": 37000.0, "filter_after_barrier_props_per_s": 35000.0}
    r["search"] = {"config3_40v_60t_arity4": {"plain": {"nodes_per_s": 1.0}, "batched": {"nodes_per_s": 2.0},
                                              "batched_device": {"nodes_per_s": 3.0}}}
    r["learned_order"] = {"scaled_family": {"summary": {"instances": 3, "learned": {
        "geomean_time_vs_first_fail": 0.6}}}}
    s = bench.summary(r)
    assert s["bulk_frac_events"] == {"t1e6": 0.1} and s["bulk_frac_of_read_ceiling"] == {"t1e6": 0.5}
    assert s["stream_1e7"] == {"props_per_s": 29000.0, "frac": 0.04}
    assert s["early_filter"] == [37000.0, 35000.0]
    assert s["config3_nodes_per_s"] == {"plain": 1.0, "batched": 2.0, "device": 3.0}
    assert s["learned_geomean_time_vs_first_fail"] == {"learned": 0.6} and "error" not in s
