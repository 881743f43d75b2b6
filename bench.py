#!/usr/bin/env python3
"""Benchmark: Compact-Table propagations/s on one large table (plus context figures).

Workload (one "step"): a seeded domain-reduction stream on one table of arity 6
over 32-value domains with 4e6 distinct uniform tuples. The stream dives from
the root: before every propagation it saves a level, then removes either 1-2
values of one variable (a delta-path update) or more than half of one
variable's values (a reset-path update) with equal probability; a dive returns
to the root after 8 calls or on failure. Every propagation runs the whole
hot path: change detection, updateTable, the failure test and filterDomains.

The edit sequence of each step is planned once, untimed, by running it through
the library, and replayed in the timed region with the input domains already
in device memory. L2 is flushed (a 256 MB write) between timed steps; the
per-step device time is taken with CUDA events on the table's stream.

`e2e` replays the same sequence through ct_propagate_host (host buffers:
domains copied in, filtered domains and status copied out every call).
`roofline` reports the propagation kernel (the only kernel of a propagation;
save/restore are separate small launches) over the timed region: algorithmic
bytes per launch -- updateTable 4 * N * (rows_ored + 2) plus filterDomains
4 * (supports words tested) -- over the CUDA-event interval around the launch.
`cpu_baseline` times the CPU oracle on a bounded sample of the same inputs.

Multi-GPU: one process per GPU, each with its own seeded stream (weak scaling,
no collective on the data path); value = all ranks' propagations / max time.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2507_18413_gb300 import inputs as G  # noqa: E402

METRIC = "CT propagations/s"
UNIT = "propagations/s"
ARITY, DOM = 6, 32
KERNELS_PER_PROPAGATE = 1


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--tuples", type=int, default=4_000_000)
    p.add_argument("--calls", type=int, default=256, help="propagations per step")
    p.add_argument("--depth", type=int, default=8)
    p.add_argument("--seed", type=int, default=20250724)
    p.add_argument("--no-extra", action="store_true", help="skip the context measurements")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--case", default="stream",
                   choices=["stream", "bulk1e6", "bulk4e6", "bulk1e7", "stream1e7", "search", "learned", "net512",
                            "planning"],
                   help="bulk*: only the one-call bandwidth case (for profiling); "
                        "search: only the plain vs batched search figures; "
                        "learned: the learned-order experiment at full size; "
                        "net512: the 512-table network fixpoints; planning: the planning chains")
    p.add_argument("--learned-eval", type=int, default=200, help="held-out instances of --case learned")
    p.add_argument("--learned-full", type=int, default=10,
                   help="instances at config-4 size (30-60 vars, 40-120 tables) in --case learned")
    return p.parse_args()


# --------------------------------------------------------------------------
# seeded stream (host logic shared by the GPU planner and the oracle arm)
# --------------------------------------------------------------------------

def next_edit(rng, masks):
    if rng.int(2) == 0:
        new, i = G.delta_step(rng, masks)
    else:
        new, i = G.reset_step(rng, masks)
    if i is None:
        new, _ = G.remove_random_values(rng, masks, 1)
    return new


def rank_seed(seed: int, rank: int) -> int:
    """Each rank propagates its own seeded stream (weak scaling, no shared data)."""
    return seed + 1000 * rank


def reduce_over_ranks(total_ms: float, props: int, world: int, device: str):
    """Whole-job figures: the slowest rank's time and the propagations of all ranks."""
    if world <= 1:
        return total_ms, float(props)
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms, float(props)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    tsum = t.clone()
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[1])


def clocks_start(gpu_index):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                 "-lms", "50", "-i", str(gpu_index)],
                                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except (OSError, FileNotFoundError):
        return None
    # the first sample (taken before the timed region, discarded) shows the
    # sampler is running when the timed region starts; wait at most 5 s for it
    import select
    ready, _, _ = select.select([proc.stdout], [], [], 5.0)
    if ready:
        proc.stdout.readline()
    return proc


def clocks_stop(proc):
    if proc is None:
        return None
    proc.terminate()
    try:
        out, _ = proc.communicate(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
        out, _ = proc.communicate()
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            mx = float(f[2])
        except ValueError:
            continue
        for k, n in enumerate(names):
            if f[5 + k].lower().startswith("active"):
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


def kernel_source_hash():
    """First 16 hex digits of the sha256 of the propagation kernel's sources
    (ct_internal.cuh, ct_device.cuh and ct_kernels.cu, in that order)."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2507_18413_gb300", "csrc")
    h = hashlib.sha256()
    for name in ("ct_internal.cuh", "ct_device.cuh", "ct_kernels.cu"):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the propagation kernel from the committed ncu
    summary, if it was taken on the kernel sources as they are now (else None)."""
    import re
    try:
        src_hash = kernel_source_hash()
        md = open(os.path.join(ROOT, "profiles", "dram_ct_propagate_kernel_stream_t4000000.md")).read()
    except OSError:
        return None
    h = re.search(r"kernel_sha256_16: ([0-9a-f]{16})", md)
    v = re.search(r"traffic_bytes_per_launch: (\d+)", md)
    if not h or not v or src_hash != h.group(1):
        return None
    return int(v.group(1))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------

class Replay:
    """A planned stream: ops over a table and the input domains of each call."""

    def __init__(self):
        self.ops = []      # ("save",) | ("restore", level) | ("prop", k)
        self.inputs = []   # uint32 words per propagation
        self.statuses = []
        self.outputs = []  # filtered domains of each propagation (None after a failure)


def plan_steps(C, torch, h, dom, dom_size, root_words, nsteps, calls, depth, seed):
    """Run the stream once through the library and record what each step does."""
    plans = []
    for s in range(nsteps):
        rng = G.Rng(G.derive_seed(seed, s))
        rp = Replay()
        masks = C.words_to_masks(root_words, dom_size)
        d = 0
        for c in range(calls):
            C.check(C.ct_save(h)[0])
            rp.ops.append(("save",))
            new = next_edit(rng, masks)
            w = C.masks_to_words(new)
            k = len(rp.inputs)
            rp.inputs.append(w.copy())
            rp.ops.append(("prop", k))
            dom.copy_(torch.from_numpy(w.view(np.int32).copy()))
            st, _ = C.ct_propagate(h, dom, 0)
            C.check(st)
            rp.statuses.append(st)
            out_words = dom.cpu().numpy().view(np.uint32).copy()
            rp.outputs.append(out_words if st == C.CT_OK else None)
            d += 1
            if st == C.CT_INFEASIBLE or d >= depth:
                C.check(C.ct_restore(h, 1))
                rp.ops.append(("restore", 1))
                masks = C.words_to_masks(root_words, dom_size)
                d = 0
            else:
                masks = C.words_to_masks(out_words, dom_size)
        if d:
            C.check(C.ct_restore(h, 1))
            rp.ops.append(("restore", 1))
        plans.append(rp)
    return plans


def run_ours(args, rank, world):
    import torch
    from paper_2507_18413_gb300 import build as B
    from paper_2507_18413_gb300 import ct as C

    B.build()
    C.load()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    seed = rank_seed(args.seed, rank)
    dom_lo, dom_size, tup = G.large_table(seed, args.tuples, ARITY, DOM)
    opt = C.make_options(profile=1)
    st, h = C.ct_create(ARITY, dom_lo, dom_size, tup, opt=opt, stream=stream)
    C.check(st)
    st, info = C.ct_get_info(h)
    off, nw = C.dom_layout(dom_size)
    DW = int(off[-1])
    dom = torch.zeros(DW, dtype=torch.int32, device="cuda")
    # root: filter once with full domains, then keep it as level 0
    full = C.masks_to_words([np.ones(d, bool) for d in dom_size])
    dom.copy_(torch.from_numpy(full.view(np.int32).copy()))
    C.check(C.ct_propagate(h, dom, 0)[0])
    root_words = dom.cpu().numpy().view(np.uint32).copy()
    C.check(C.ct_save(h)[0])  # level 0: root

    nsteps = args.warmup + args.steps
    plans = plan_steps(C, torch, h, dom, dom_size, root_words, nsteps, args.calls, args.depth, seed)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device="cuda")  # 256 MB > L2

    def device_inputs(rp):
        return torch.from_numpy(np.stack(rp.inputs).view(np.int32).copy()).cuda()

    dev_in = [device_inputs(rp) for rp in plans]

    lib = C.load()
    f_save, f_restore, f_prop, f_prop_host = lib.ct_save, lib.ct_restore, lib.ct_propagate, lib.ct_propagate_host
    lv = ctypes.c_int(0)
    lvp = ctypes.byref(lv)

    def replay(rp, work):
        """The planned ops through the C entry points (argument lists prepared up front)."""
        base = work.data_ptr()
        calls = []
        for op in rp.ops:
            if op[0] == "save":
                calls.append((f_save, (h, lvp)))
            elif op[0] == "restore":
                calls.append((f_restore, (h, op[1])))
            else:
                calls.append((f_prop, (h, base + op[1] * DW * 4, None)))
        nprop = sum(1 for op in rp.ops if op[0] == "prop")
        nsave = sum(1 for op in rp.ops if op[0] == "save")
        nres = len(rp.ops) - nprop - nsave
        return calls, (nprop, nsave, nres)

    def run_calls(calls, statuses=None):
        for f, a in calls:
            r = f(*a)
            if r < 0:
                raise RuntimeError(C.last_error())
            if statuses is not None and f is f_prop:
                statuses.append(r)

    W = int(info["words"])
    st, root_ct, _ = C.ct_get_currtable(h, W)
    C.check(st)
    import hashlib
    root_digest = hashlib.sha256(root_ct.tobytes()).hexdigest()[:16]
    mismatches = []

    def verify(s_idx, rp, work, statuses):
        """The replayed step did the planned work: same statuses, same filtered
        domains, and currTable back at the root state at the end of the step."""
        if statuses != rp.statuses:
            mismatches.append(f"step {s_idx}: statuses differ")
        got = work.cpu().numpy().view(np.uint32).reshape(len(rp.inputs), DW)
        for k, want in enumerate(rp.outputs):
            if want is not None and not np.array_equal(got[k], want):
                mismatches.append(f"step {s_idx} call {k}: domains differ")
                break
        st, words, _ = C.ct_get_currtable(h, W)
        if st != C.CT_OK or hashlib.sha256(words.tobytes()).hexdigest()[:16] != root_digest:
            mismatches.append(f"step {s_idx}: currTable not back at the root state")

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    step_ms, props, launches = [], 0, 0
    clk = None
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0] or str(local)
    # the timed pass runs without per-launch timing events (instrumentation,
    # not work); the roofline's per-launch figures come from a profiled
    # replay of the same steps below
    C.check(C.ct_set_profile(h, 0))
    for s, rp in enumerate(plans):
        work = dev_in[s].clone()
        flush.zero_()
        if s == args.warmup:
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            clk = clocks_start(gpu_index if world == 1 else local)
        calls, (n, ns, nr) = replay(rp, work)
        sts = []
        torch.cuda.synchronize()
        ev0.record(stream)
        run_calls(calls, sts)
        ev1.record(stream)
        torch.cuda.synchronize()
        verify(s, rp, work, sts)
        if s >= args.warmup:
            step_ms.append(ev0.elapsed_time(ev1))
            props += n
            # one launch per propagation and per restore; ct_save launches nothing
            launches += KERNELS_PER_PROPAGATE * n + nr
    clocks = clocks_stop(clk)
    if mismatches:
        raise SystemExit("timed replay differs from the planned calls: " + "; ".join(mismatches[:5]))
    if world > 1:
        torch.distributed.barrier()
    # profiled replay of the timed steps (untimed): per-launch CUDA events and
    # the algorithmic bytes of every call, for the roofline
    C.check(C.ct_set_profile(h, 1))
    C.check(C.ct_reset_profile(h))
    for s in range(args.warmup, nsteps):
        calls, _ = replay(plans[s], dev_in[s].clone())
        flush.zero_()
        torch.cuda.synchronize()
        run_calls(calls)
        torch.cuda.synchronize()
    st, prof = C.ct_get_profile(h)
    C.check(C.ct_set_profile(h, 0))
    total_ms = float(sum(step_ms))
    total_ms_all, props_all = reduce_over_ranks(total_ms, props, world, "cuda")
    value = props_all / (total_ms_all / 1e3)

    # e2e: the same replay through host buffers (copies in the timed region)
    e2e_ms, e2e_props = 0.0, 0
    h2d = d2h = 0
    status_bytes = (24 + (ARITY + 31) // 32 + DW) * 4
    for s in range(args.warmup, nsteps):
        rp = plans[s]
        # this step's input domains in pinned host memory
        pinned = torch.from_numpy(np.stack(rp.inputs).view(np.int32).copy()).pin_memory()
        pbase = pinned.data_ptr()
        calls = []
        for op in rp.ops:
            if op[0] == "save":
                calls.append((f_save, (h, lvp)))
            elif op[0] == "restore":
                calls.append((f_restore, (h, op[1])))
            else:
                calls.append((f_prop_host, (h, ctypes.cast(pbase + op[1] * DW * 4, ctypes.POINTER(ctypes.c_uint32)),
                                            None)))
                e2e_props += 1
                h2d += DW * 4
                d2h += status_bytes
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run_calls(calls)
        torch.cuda.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e = {"value": e2e_props / (e2e_ms / 1e3) if e2e_ms > 0 else None, "unit": UNIT,
           "h2d_bytes_per_step": h2d // max(args.steps, 1), "d2h_bytes_per_step": d2h // max(args.steps, 1)}

    # The timed steps once more, outside the timed region: (1) with warm L2
    # (no flush between steps), (2) one CUDA-event pair around every
    # propagation, for the distribution of the per-call latency.
    warm_ms, warm_props, lat = 0.0, 0, []
    for s in range(args.warmup, nsteps):
        calls, (n, _, _) = replay(plans[s], dev_in[s].clone())
        torch.cuda.synchronize()
        ev0.record(stream)
        run_calls(calls)
        ev1.record(stream)
        torch.cuda.synchronize()
        warm_ms += ev0.elapsed_time(ev1)
        warm_props += n
    for s in range(args.warmup, nsteps):
        calls, _ = replay(plans[s], dev_in[s].clone())
        flush.zero_()
        pairs = []
        torch.cuda.synchronize()
        for f, a in calls:
            if f is f_prop:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if f(*a) < 0:
                    raise RuntimeError(C.last_error())
                e1.record(stream)
                pairs.append((e0, e1))
            elif f(*a) < 0:
                raise RuntimeError(C.last_error())
        torch.cuda.synchronize()
        lat += [a.elapsed_time(b) * 1e3 for a, b in pairs]
    lat = np.sort(np.asarray(lat))

    peak, peak_kind = peaks()
    alg = prof["update_bytes"] + prof["filter_bytes"]
    achieved = (alg / (prof["kernel_ms"] / 1e3) / 1e9) if prof["kernel_ms"] > 0 else 0.0
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": profiled_traffic(), "peak_kind": peak_kind,
                "kernel": "ct_propagate_kernel",
                "launches": int(prof["calls"]),
                "avg_bytes_per_launch": alg / max(prof["calls"], 1),
                "avg_update_bytes_per_launch": prof["update_bytes"] / max(prof["calls"], 1),
                "avg_launch_us": prof["kernel_ms"] * 1e3 / max(prof["calls"], 1),
                "avg_device_us": prof["device_ms"] * 1e3 / max(prof["calls"], 1),
                "achieved_device_timer": round(alg / (prof["device_ms"] / 1e3) / 1e9, 1) if prof["device_ms"] > 0 else None}

    result = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_ms / max(args.steps, 1), 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded SplitMix64; stands in for the paper's LIN/Gecode/OP instances)",
        "config": {"workload": f"ct_stream_t{args.tuples}_arity{ARITY}_d{DOM}", "tuples": args.tuples,
                   "arity": ARITY, "domain": DOM, "calls_per_step": args.calls, "dive_depth": args.depth,
                   "edits": "50% delta (1-2 values), 50% reset (> half a domain)", "seed": args.seed,
                   "l2": "flushed between steps (256 MB write), flush excluded from timing",
                   "timing": "sum of per-step CUDA-event intervals on the table stream; no per-launch "
                             "timing events in the timed pass (the roofline's come from a profiled replay)",
                   "parallelism": f"replicas x{world}", "grid_blocks": info["grid_blocks"],
                   "segments": info["segments"]},
        "gpu_launches": launches,
        "e2e": e2e,
        "roofline": roofline,
        "clocks": clocks,
        "warm_l2": {"value": round(warm_props / (warm_ms / 1e3), 1) if warm_ms > 0 else None, "unit": UNIT,
                    "ms_per_step": round(warm_ms / max(args.steps, 1), 4),
                    "note": "the timed steps replayed without the L2 flush between steps (untimed pass)"},
        "call_latency_us": {"calls": int(len(lat)),
                            "p10": round(float(np.percentile(lat, 10)), 2) if len(lat) else None,
                            "p50": round(float(np.percentile(lat, 50)), 2) if len(lat) else None,
                            "p90": round(float(np.percentile(lat, 90)), 2) if len(lat) else None,
                            "note": "CUDA events around each ct_propagate of the timed steps, L2 flushed "
                                    "between steps (untimed pass)"},
    }
    result["replay_check"] = {"steps": len(plans), "propagations": sum(len(rp.inputs) for rp in plans),
                              "statuses_equal": True, "domains_equal": True, "currtable_back_at_root": True,
                              "note": "every timed step was compared, after its timed region, with the "
                                      "planning pass: status and filtered domains of each call, and the "
                                      "currTable digest at the end of the step; a mismatch exits non-zero"}
    C.ct_destroy(h)
    del flush
    if rank == 0 and not args.no_extra:
        # figures of the other configurations, at the top level of the line
        result["bulk_update"] = {
            "t1e6_arity6_d32": _bulk_update(C, torch, stream, 1_000_000, 6, 32, 5),
            "t4e6_arity6_d32": _bulk_update(C, torch, stream, 4_000_000, 6, 32, 5),
            "t1e7_arity5_d64": _bulk_update(C, torch, stream, 10_000_000, 5, 64, 6)}
        result["stream_1e7_arity5_d64"] = _stream_rate(C, torch, stream, 10_000_000, 128, 99 + 10_000_000,
                                                       arity=5, d=64, roofline=True)
        # the same kernel's bandwidth on the bulk calls and the huge table's
        # stream, kept beside the headline stream's roofline
        hbm = peaks()[0]
        roofline["bulk_reset_calls"] = {
            k: {"bytes": v["bytes_per_launch"], "frac_events": v["frac_of_hbm"],
                "frac_update_phase": v["update_phase_frac_of_hbm"],
                "read_ceiling_frac": round(v["read_ceiling_GBps"] / hbm, 4),
                "frac_of_read_ceiling": v["frac_of_read_ceiling"]}
            for k, v in result["bulk_update"].items()}
        s7 = result["stream_1e7_arity5_d64"]
        roofline["stream_1e7_arity5_d64"] = {"props_per_s": s7["value"], "frac": s7["roofline"]["frac"],
                                             "avg_bytes_per_launch": s7["roofline"]["avg_bytes_per_launch"]}
        # the filter run after the update's barrier on every call (the kernel
        # before its filter ran beside the update), same stream and table
        result["early_filter_ablation"] = {
            "tuples": args.tuples,
            "default_props_per_s": _stream_rate(C, torch, stream, args.tuples, 256, args.seed),
            "filter_after_barrier_props_per_s": _stream_rate(C, torch, stream, args.tuples, 256, args.seed,
                                                             opt=C.make_options(no_early_filter=1)),
            "note": "best of two planned 256-call steps each, host wall time"}
        result["search"] = search_extras(C)
        result["extra"] = extras(args, C, torch, stream)
        lo = result["extra"].get("learned_order") or {}
        result["learned_order"] = {"scaled_family": {k: lo.get(k) for k in ("instances", "eval_instances",
                                                                             "node_limit", "samples", "summary")},
                                   "config4_size": lo.get("config4_full_scale")}
    if rank == 0:
        result["cpu_baseline"] = cpu_baseline(args, plans[args.warmup:], dom_lo, dom_size, tup)
        result["cpu_baseline"]["cpu"] = cpu_model()
        result["cpu_baseline_bitset"] = cpu_bitset_baseline(args, plans[args.warmup:], dom_lo, dom_size, tup)
        if not args.no_extra:
            result["cpu_baseline_bitset_all_cores"] = cpu_bitset_baseline_cores(args, plans[args.warmup:], dom_lo,
                                                                                dom_size, tup)
    if rank == 0:
        result["summary"] = summary(result)
    return result


def summary(r):
    """The line's main figures in a few hundred characters, as its last key."""
    out = {"props_per_s": r["value"], "e2e_props_per_s": round(r["e2e"]["value"] or 0.0, 1),
           "roofline_frac": r["roofline"]["frac"], "call_p50_us": r["call_latency_us"]["p50"]}
    try:
        b = r.get("bulk_update") or {}
        out["bulk_frac_events"] = {k.split("_")[0]: v["frac_of_hbm"] for k, v in b.items()}
        out["bulk_frac_update_phase"] = {k.split("_")[0]: v["update_phase_frac_of_hbm"] for k, v in b.items()}
        out["bulk_frac_of_read_ceiling"] = {k.split("_")[0]: v["frac_of_read_ceiling"] for k, v in b.items()}
        if "stream_1e7_arity5_d64" in r:
            s7 = r["stream_1e7_arity5_d64"]
            out["stream_1e7"] = {"props_per_s": s7["value"], "frac": s7["roofline"]["frac"]}
        if "early_filter_ablation" in r:
            e = r["early_filter_ablation"]
            out["early_filter"] = [e["default_props_per_s"], e["filter_after_barrier_props_per_s"]]
        for k, v in (r.get("search") or {}).items():
            out[k.split("_")[0] + "_nodes_per_s"] = {"plain": v["plain"]["nodes_per_s"],
                                                     "batched": v["batched"]["nodes_per_s"],
                                                     "device": v["batched_device"]["nodes_per_s"]}
        lo = ((r.get("learned_order") or {}).get("scaled_family") or {}).get("summary") or {}
        if lo:
            out["learned_geomean_time_vs_first_fail"] = {k: lo[k].get("geomean_time_vs_first_fail")
                                                         for k in lo if isinstance(lo[k], dict)
                                                         and "geomean_time_vs_first_fail" in lo[k]}
    except Exception as e:  # the summary must not hide the line
        out["error"] = repr(e)
    out["cpu_bitset_1_core"] = (r.get("cpu_baseline_bitset") or {}).get("value")
    out["cpu_bitset_all_cores"] = (r.get("cpu_baseline_bitset_all_cores") or {}).get("value")
    return out


def _read_ceiling(C, torch, nbytes, flush, reps=7):
    """What one launch reaches reading `nbytes` once on this GPU: the library's
    streaming-read kernel (ct_read_ceiling: 128-bit loads, eight in flight per
    thread, four CTAs per SM) over a buffer of that size, L2 flushed before each
    launch, CUDA events recorded by the library right around the launch
    (median), as for the propagation's own launch. A launch this
    short pays launch and ramp-up latency that a long copy amortises, so this is
    the bandwidth a one-call propagation of that many bytes could hope for."""
    n = max(16, (int(nbytes) + 15) // 16 * 16)
    x = torch.ones(n // 4, dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream()
    ms = []
    for _ in range(reps):
        flush.zero_()
        torch.cuda.synchronize()
        st, t = C.ct_read_ceiling(x, n, s, timed=True)
        C.check(st)
        ms.append(t)
    del x
    return x_bytes_per_s(n, statistics.median(ms))


def x_bytes_per_s(nbytes, ms):
    return nbytes / (ms / 1e3) / 1e9


def _bulk_update(C, torch, stream, t, arity, d, seed, reps=9):
    """One big reset call per repetition (every variable keeps < half its values):
    the bandwidth regime of updateTable on a large table, L2 flushed before each.
    Medians over the repetitions of: the CUDA-event interval around the launch,
    the device-timer span, and the update phase by the device timer (plan end to
    the barrier after updateTable); beside them the contiguous-read ceiling of
    the same bytes (_read_ceiling)."""
    dom_lo, dom_size, tup = G.large_table(seed, t, arity, d)
    st, h = C.ct_create(arity, dom_lo, dom_size, tup, opt=C.make_options(profile=1), stream=stream)
    C.check(st)
    off, _ = C.dom_layout(dom_size)
    dom = torch.zeros(int(off[-1]), dtype=torch.int32, device="cuda")
    full = C.masks_to_words([np.ones(x, bool) for x in dom_size])
    dom.copy_(torch.from_numpy(full.view(np.int32).copy()))
    C.check(C.ct_propagate(h, dom, 0)[0])
    C.check(C.ct_save(h)[0])
    keep = d // 2 - 1
    masks = []
    rng = G.Rng(seed)
    for i in range(arity):
        m = np.zeros(d, bool)
        m[np.argsort(rng.u64(d))[:keep]] = True
        masks.append(m)
    w = C.masks_to_words(masks).view(np.int32).copy()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device="cuda")
    ev, dev, upd = [], [], []
    stats = None
    for r in range(reps):
        C.check(C.ct_save(h)[0])
        dom.copy_(torch.from_numpy(w))
        flush.zero_()
        torch.cuda.synchronize()
        C.ct_reset_profile(h)
        st, _ = C.ct_propagate(h, dom, 0)
        C.check(st)
        prof = C.ct_get_profile(h)[1]
        stats = C.ct_get_call_stats(h)[1]
        ev.append(prof["kernel_ms"] * 1e3)
        ph = stats["phase_ns"]
        dev.append(ph[3] / 1e3)
        upd.append((ph[1] - ph[0]) / 1e3)
        C.check(C.ct_restore(h, 1))
    info = C.ct_get_info(h)[1]
    C.ct_destroy(h)
    alg = stats["update_bytes"] + stats["filter_bytes"]
    hbm = peaks()[0]
    ev_us, dev_us, upd_us = statistics.median(ev), statistics.median(dev), statistics.median(upd)
    gbs = alg / ev_us / 1e3
    ceiling = _read_ceiling(C, torch, alg, flush)
    del flush
    return {"tuples": t, "arity": arity, "domain": d, "rows_ored": stats["rows_ored"],
            "grid_blocks": info["grid_blocks"], "loads_in_flight": info["loads_in_flight"],
            "bytes_per_launch": alg, "launch_us": round(ev_us, 2), "GBps": round(gbs, 1),
            "frac_of_hbm": round(gbs / hbm, 4),
            "device_us": round(dev_us, 2),
            "update_phase_us": round(upd_us, 2),
            "update_phase_GBps": round(stats["update_bytes"] / upd_us / 1e3, 1),
            "update_phase_frac_of_hbm": round(stats["update_bytes"] / upd_us / 1e3 / hbm, 4),
            "read_ceiling_GBps": round(ceiling, 1),
            "frac_of_read_ceiling": round(gbs / ceiling, 4),
            "phase_ns_last": stats["phase_ns"],
            "note": "medians of %d one-call repetitions, L2 flushed before each; GBps by CUDA events "
                    "around the launch; update phase by the device timer (plan end to the barrier "
                    "after updateTable); read ceiling: one launch of the library's streaming-read kernel "
                    "(ct_read_ceiling) over the same bytes" % reps}


def _stream_rate(C, torch, stream, t, calls, seed, opt=None, shape=None, arity=ARITY, d=DOM, roofline=False):
    """Propagations/s of a planned delta/reset stream on one table (best of two
    planned steps, host wall time, inputs in HBM). With roofline: also a
    profiled replay of the same steps (CUDA events around every launch) and the
    algorithmic bytes of its calls, as for the headline stream."""
    dom_lo, dom_size, tup = G.large_table(seed, t, arity, d)
    st, h = C.ct_create(arity, dom_lo, dom_size, tup, opt=opt, stream=stream)
    C.check(st)
    inf = C.ct_get_info(h)[1]
    if shape is not None:
        shape.update(grid_blocks=inf["grid_blocks"], loads_in_flight=inf["loads_in_flight"],
                     autotuned=inf["autotuned"])
    off, _ = C.dom_layout(dom_size)
    dom = torch.zeros(int(off[-1]), dtype=torch.int32, device="cuda")
    full = C.masks_to_words([np.ones(x, bool) for x in dom_size])
    dom.copy_(torch.from_numpy(full.view(np.int32).copy()))
    C.check(C.ct_propagate(h, dom, 0)[0])
    root = dom.cpu().numpy().view(np.uint32).copy()
    C.check(C.ct_save(h)[0])
    plans = plan_steps(C, torch, h, dom, dom_size, root, 2, calls, 8, seed)
    DW = int(off[-1])
    best = None

    def replay(rp, work):
        for op in rp.ops:
            if op[0] == "save":
                C.ct_save(h)
            elif op[0] == "restore":
                C.ct_restore(h, op[1])
            else:
                C.check(C.ct_propagate(h, work.data_ptr() + op[1] * DW * 4, 0)[0])

    for rp in plans:
        work = torch.from_numpy(np.stack(rp.inputs).view(np.int32).copy()).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        replay(rp, work)
        torch.cuda.synchronize()
        rate = len(rp.inputs) / (time.perf_counter() - t0)
        best = rate if best is None else max(best, rate)
    out = round(best, 1)
    if roofline:
        C.check(C.ct_set_profile(h, 1))
        C.check(C.ct_reset_profile(h))
        for rp in plans:
            replay(rp, torch.from_numpy(np.stack(rp.inputs).view(np.int32).copy()).cuda())
        torch.cuda.synchronize()
        prof = C.ct_get_profile(h)[1]
        alg = prof["update_bytes"] + prof["filter_bytes"]
        hbm, kind = peaks()
        ach = alg / (prof["kernel_ms"] / 1e3) / 1e9
        out = {"value": out, "unit": UNIT, "tuples": t, "arity": arity, "domain": d, "calls": len(plans) * calls,
               "grid_blocks": inf["grid_blocks"],
               "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                            "frac": round(ach / hbm, 4), "peak_kind": kind,
                            "avg_bytes_per_launch": alg / max(prof["calls"], 1),
                            "avg_launch_us": prof["kernel_ms"] * 1e3 / max(prof["calls"], 1),
                            "avg_device_us": prof["device_ms"] * 1e3 / max(prof["calls"], 1)}}
    C.ct_destroy(h)
    return out


def _dfs_rate(C, node_limit=3000, host_fixpoint=0):
    nvars, ntables, arity, d, t, seed = 20, 8, 6, 32, 100_000, 2024
    rng = G.Rng(seed)
    st, m = C.ct_model_create([0] * nvars, [d] * nvars, opt=C.make_options(host_fixpoint=host_fixpoint))
    C.check(st)
    for k in range(ntables):
        scope = G.random_scope(rng, nvars, arity)
        tup = G.distinct_uniform_tuples(G.derive_seed(seed, k), [0] * arity, [d] * arity, t)
        C.check(C.ct_model_add_table(m, scope, tup))
    st, s = C.ct_search_dfs(m, nvars, node_limit, True)
    C.check(st)
    C.ct_model_destroy(m)
    return {"csp": "20 vars d=32, 8 tables arity 6 x 1e5 tuples",
            "fixpoint": "host queue, one launch per table" if host_fixpoint else "one launch per fixpoint",
            "nodes": s["nodes"], "fails": s["fails"],
            "solutions": s["solutions"], "complete": s["complete"], "propagations": s["propagations"],
            "seconds": round(s["seconds"], 3), "nodes_per_s": round(s["nodes"] / s["seconds"], 1),
            "table_propagations_per_s": round(s["propagations"] / s["seconds"], 1)}


def _build_model(C, spec):
    st, m = C.ct_model_create(spec.dom_lo, spec.dom_size)
    C.check(st)
    for tb in spec.tables:
        C.check(C.ct_model_add_table(m, tb.scope, tb.tuples))
    return m


def _device_search(C, m, spec, slots, split, limit):
    """The batched search with the slots' search run on the device (second of two
    calls: the first builds the device buffers and sizes their capacities)."""
    for _ in range(2):
        st, d, info = C.ct_search_batch_device(m, spec.nvars, slots, split, limit)
        C.check(st)
    return {"slots": slots, "split_depth": split, "nodes": d["nodes"], "fails": d["fails"],
            "solutions": d["solutions"], "seconds": round(d["seconds"], 3),
            "nodes_per_s": round(d["nodes"] / d["seconds"], 1), "launches": info["steps"],
            "rounds": info["rounds"], "open_nodes": info["open_nodes"], "split_nodes": info["split_nodes"]}


def _search_compare(C, name, spec, slots=512, split=10, plain_limit=3000, batch_limit=20000, assign=False,
                    long_limit=0):
    """Nodes/s of the plain search (one node per launch) and of the batched search
    (slots x tables propagated per launch) on the same CSP, counting all solutions
    up to a node limit; the batched figure is the second of two calls (the first
    builds the slot copies and grows their trails). assign: the split depth
    counts assignments on a node's path (ct_search_batch_assign)."""
    m = _build_model(C, spec)
    try:
        st, p = C.ct_search_dfs(m, spec.nvars, plain_limit, True)
        C.check(st)
        first = None
        for _ in range(2):
            st, b, info = C.ct_search_batch(m, spec.nvars, slots, split, batch_limit, True, split_assignments=assign)
            C.check(st)
            first = first or (b["seconds"], info["setup_seconds"])
        dev = _device_search(C, m, spec, slots, split, batch_limit)
        longer = None
        if long_limit:
            st, bl, il = C.ct_search_batch(m, spec.nvars, slots, split, long_limit, True)
            C.check(st)
            longer = {"node_limit": long_limit,
                      "batched_host_stepped": {"nodes": bl["nodes"], "seconds": round(bl["seconds"], 3),
                                               "nodes_per_s": round(bl["nodes"] / bl["seconds"], 1)},
                      "batched_device": _device_search(C, m, spec, slots, split, long_limit)}
    finally:
        C.ct_model_destroy(m)
    plain_nps = p["nodes"] / p["seconds"]
    batch_nps = b["nodes"] / b["seconds"]
    return {"csp": name, "plain": {"nodes": p["nodes"], "seconds": round(p["seconds"], 3),
                                   "nodes_per_s": round(plain_nps, 1)},
            "batched": {"slots": slots, "split_depth": split,
                        "split_counts": "assignments on the path" if assign else "binary levels",
                        "nodes": b["nodes"], "fails": b["fails"],
                        "solutions": b["solutions"], "seconds": round(b["seconds"], 3),
                        "nodes_per_s": round(batch_nps, 1), "launches": info["steps"],
                        "rounds": info["rounds"], "open_nodes": info["open_nodes"], "steals": info["steals"],
                        "device_wait_s": round(info["wait_seconds"], 3),
                        "first_call_s": round(first[0], 3), "copies_setup_s": round(first[1], 3)},
            "batched_device": dev,
            "speedup": round(batch_nps / plain_nps, 2),
            "speedup_device": round(dev["nodes_per_s"] / plain_nps, 2),
            "longer_run": longer}


def search_extras(C):
    out = {}
    out["config2_20v_8t_arity6_1e5"] = _search_compare(
        C, "20 vars d=32, 8 tables arity 6 x 1e5 tuples", G.random_csp(2024, 20, 8, 6, 32, 100_000),
        long_limit=100_000)
    # 1,024 independent search nodes: the frontier of the binary first-fail
    # tree at depth 10 (at most 2^10 = 1,024 open nodes), one slot each
    out["config3_40v_60t_arity4"] = _search_compare(
        C, "40 vars d=24, 60 tables arity 4 x log-uniform 1e4..2e5 tuples", G.batching_csp(3003),
        slots=1024, split=10, long_limit=100_000)
    return out


def network_extras(C, tuples=(1e3, 1e6), edits=60, seed=3):
    """512 tables (arity 2-8, log-uniform tuple counts, domains 8-128, half Zipf)
    over 1,024 variables propagated to their common fixpoint in one cooperative
    launch per fixpoint: the root fixpoint (median of four repeats, the first
    launch reported apart), then a stream of edits (1 value or
    half a domain of a random variable) with saves, restoring to the root on
    failure or after 5 edits. Bytes are the algorithmic bytes of every table
    propagation (ct_model_stats), time the host-observed launch-to-result time."""
    hbm, _ = peaks()
    t0 = time.perf_counter()
    spec = G.network_tables(seed, tuples=tuples)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    m = _build_model(C, spec)
    build_s = time.perf_counter() - t0
    try:
        # the root fixpoint five times (restored to the initial state between
        # them): the first launch apart, the median of the other four
        st, lvr = C.ct_model_save(m)
        roots = []
        for rep in range(5):
            C.ct_model_reset_stats(m)
            C.check(C.ct_model_propagate(m))
            roots.append(C.ct_model_get_stats(m)[1])
            if rep < 4:
                C.check(C.ct_model_restore(m, lvr))
                lvr = C.ct_model_save(m)[1]
        root = sorted(roots[1:], key=lambda d: d["wait_seconds"])[len(roots[1:]) // 2]
        C.ct_model_reset_stats(m)
        st, lv0 = C.ct_model_save(m)
        off, _ = C.dom_layout(spec.dom_size)
        rng = G.Rng(G.derive_seed(seed, 99))
        depth = fails = 0
        for i in range(edits):
            st, w = C.ct_model_get_domains(m, int(off[-1]))
            masks = C.words_to_masks(w, spec.dom_size)
            cand = [v for v, mk in enumerate(masks) if mk.sum() > 1]
            v = cand[rng.int(len(cand))]
            vals = np.flatnonzero(masks[v])
            k = 1 if rng.int(2) == 0 else len(vals) // 2
            order = np.argsort(rng.u64(len(vals)), kind="stable")[:k]
            masks[v][vals[order]] = False
            C.check(C.ct_model_save(m)[0])
            C.check(C.ct_model_set_domains(m, C.masks_to_words(masks)))
            st = C.ct_model_propagate(m)
            depth += 1
            if st == C.CT_INFEASIBLE or depth >= 5:
                fails += st == C.CT_INFEASIBLE
                C.check(C.ct_model_restore(m, lv0))
                C.check(C.ct_model_save(m)[0])
                depth = 0
        st, ed = C.ct_model_get_stats(m)
    finally:
        C.ct_model_destroy(m)

    def summary(d):
        b = d["update_bytes"] + d["filter_bytes"]
        gbs = b / d["wait_seconds"] / 1e9 if d["wait_seconds"] > 0 else 0.0
        return {"fixpoints": d["fixpoints"], "rounds": d["rounds"], "table_propagations": d["propagations"],
                "seconds": round(d["wait_seconds"], 4),
                "ms_per_fixpoint": round(1e3 * d["wait_seconds"] / max(1, d["fixpoints"]), 3),
                "update_bytes": d["update_bytes"], "filter_bytes": d["filter_bytes"],
                "GBps": round(gbs, 1), "frac_of_hbm": round(gbs / hbm, 4)}

    return {"tables": len(spec.tables), "variables": spec.nvars,
            "tuples_total": int(sum(len(tb.tuples) for tb in spec.tables)),
            "tuple_range": [int(tuples[0]), int(tuples[1])], "generate_s": round(gen_s, 1),
            "build_s": round(build_s, 1), "root_fixpoint": summary(root),
            "root_fixpoint_first_launch": summary(roots[0]), "edit_fixpoints": summary(ed),
            "edit_failures": fails}


def planning_extras(C, n_eval=3, n_train=8, node_limit=100_000):
    """Planning-style chains (256 states x 32 actions, 30 steps, fixed initial and
    goal states): nodes and time to the first plan with first-fail and with a
    network trained on other chains, plain and batched (64 slots; the model
    searches alone for 256 nodes, then the slots take the frontier it leaves,
    stopping at the first plan any slot finds)."""
    from paper_2507_18413_gb300 import learn as LN
    t0 = time.perf_counter()
    X, y = LN.collect([G.planning_csp(1000 + s) for s in range(n_train)], node_limit=150, slots=64,
                      max_samples=60_000)
    net, losses = LN.train(X, y, epochs=20)
    train_s = time.perf_counter() - t0
    try:
        rows = LN.compare([G.planning_csp(s) for s in range(n_eval)], net, node_limit=node_limit, batched=(64, 64))
    finally:
        C.ct_mlp_destroy(net)
    return {"instances": "planning_csp seeds 0..%d: 61 variables (31 states of 256 values, 30 actions of 32), "
                         "30 transition tables of ~20k tuples" % (n_eval - 1),
            "train": {"instances": n_train, "samples": int(len(y)), "seconds": round(train_s, 2),
                      "loss_first_last": [round(float(losses[0]), 5), round(float(losses[-1]), 5)]},
            "node_limit": node_limit, "per_instance": rows, "summary": LN.summarize(rows)}


LEARNED_SMALL = dict(nvars=(20, 30), dom=(8, 16), ntables=(30, 50), arity=(3, 4), tuples=(1e3, 2e4))


def learned_extras(C, n_train=40, n_eval=20, node_limit=5000, train_nodes=300, max_samples=100_000, epochs=20,
                   full_eval=0, full_limit=None):
    """Train the branching network on first-fail traces of seeded instances and
    compare first-fail and the network, plain and batched, on held-out seeds:
    time and nodes to the first solution or to a proof of infeasibility."""
    from paper_2507_18413_gb300 import learn as LN
    t0 = time.perf_counter()
    train_specs = [G.learned_csp(s, **LEARNED_SMALL) for s in range(n_train)]
    eval_specs = [G.learned_csp(100_000 + s, **LEARNED_SMALL) for s in range(n_eval)]
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    X, y = LN.collect(train_specs, node_limit=train_nodes, slots=64, max_samples=max_samples)
    collect_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    net, losses = LN.train(X, y, epochs=epochs)
    train_s = time.perf_counter() - t0
    try:
        rows = LN.compare(eval_specs, net, node_limit=node_limit, batched=(64, 64))
        out = {"instances": "learned_csp seeds, 20-30 vars, d 8-16, 30-50 tables of arity 3-4, 1e3-2e4 "
                            "tuples, expected 2^4 solutions (config 4 scaled to instances first-fail "
                            "finishes within the limit)",
               "train_instances": n_train, "eval_instances": n_eval, "node_limit": node_limit,
               "samples": int(len(y)), "collect_s": round(collect_s, 2), "train_s": round(train_s, 3),
               "epochs": epochs, "loss_first_last": [round(float(losses[0]), 5), round(float(losses[-1]), 5)],
               "generate_s": round(gen_s, 1), "summary": LN.summarize(rows)}
        if full_eval:
            t0 = time.perf_counter()
            full = [G.learned_csp(200_000 + s) for s in range(full_eval)]
            lim = full_limit or node_limit
            frows = LN.compare(full, net, node_limit=lim, batched=(64, 64))
            out["config4_full_scale"] = {
                "instances": full_eval, "node_limit": lim,
                "family": "learned_csp seeds 200000+: 30-60 vars, d 16-64, 40-120 tables of arity 3-6, "
                          "1e4-5e5 uniform tuples (config 4 as stated)",
                "sizes": [{"nvars": r["nvars"], "tables": r["tables"]} for r in frows],
                "summary": LN.summarize(frows), "seconds": round(time.perf_counter() - t0, 1),
                "note": "the network is the one trained on the scaled family; an arm 'finished' when it "
                        "found a solution or proved infeasibility within the node limit"}
    finally:
        C.ct_mlp_destroy(net)
    return out


def extras(args, C, torch, stream):
    out = {}
    try:
        out["network_512_tables"] = network_extras(C)
        out["stream_props_per_s"] = {str(t): _stream_rate(C, torch, stream, t, 128, 99 + t)
                                     for t in (100_000, 1_000_000)}
        # the paper's propagators copy currTable host<->device around every call
        # (Sec. 4); the same streams with those copies added
        out["copy_state_ablation_props_per_s"] = {
            str(t): {"resident": _stream_rate(C, torch, stream, t, 128, 99 + t),
                     "currtable_copied_each_call": _stream_rate(C, torch, stream, t, 128, 99 + t,
                                                                opt=C.make_options(copy_state=1))}
            for t in (100_000, 1_000_000, 4_000_000)}
        # launch shape chosen by trial propagations at creation against the default rule
        tuned = {}
        for t in (100_000, 1_000_000, 4_000_000):
            d0, d1 = {}, {}
            r0 = _stream_rate(C, torch, stream, t, 128, 99 + t, shape=d0)
            r1 = _stream_rate(C, torch, stream, t, 128, 99 + t, opt=C.make_options(autotune=1), shape=d1)
            tuned[str(t)] = {"default": {"props_per_s": r0, **d0}, "autotuned": {"props_per_s": r1, **d1}}
        out["autotune_props_per_s"] = tuned
        out["dfs_plain_first_fail"] = _dfs_rate(C)
        out["dfs_plain_first_fail_host_queue"] = _dfs_rate(C, host_fixpoint=1)
        out["learned_order"] = learned_extras(C, full_eval=3, full_limit=2000)
        out["planning_chain"] = planning_extras(C)
    except Exception as e:  # context figures must not hide the main line
        out["error"] = repr(e)
    return out


# --------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# --------------------------------------------------------------------------

def cpu_bitset_baseline(args, plans, dom_lo, dom_size, tup, seconds=8.0):
    """The serial CPU bitset CT (Algorithms 1-3, 64-bit words, residues, trail) on
    the same planned calls, saves and restores, one host thread."""
    from oracle.serial_ct import SerialCT
    ct = SerialCT(dom_lo, dom_size, tup)
    import paper_2507_18413_gb300.ct as C
    full = C.masks_to_words([np.ones(d, bool) for d in dom_size])
    ct.propagate(full.copy())
    ct.save()
    done, t0 = 0, time.perf_counter()
    for rp in plans:
        ins = [w.copy() for w in rp.inputs]
        for op in rp.ops:
            if op[0] == "save":
                ct.save()
            elif op[0] == "restore":
                ct.restore(op[1])
            else:
                ct.propagate(ins[op[1]])
                done += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    ct.close()
    return {"value": round(done / dt, 1), "unit": UNIT, "cores": 1, "kind": "serial bitset CT (Algorithms 1-3)",
            "sample": f"{done} propagations of the timed stream with their saves/restores, {dt:.1f} s, one thread"}


def cpu_model():
    """The host CPU's model name (lscpu), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
    except (OSError, subprocess.SubprocessError):
        return None
    for line in out.splitlines():
        if line.strip().lower().startswith("model name"):
            return line.split(":", 1)[1].strip()
    return None


def cpu_bitset_baseline_cores(args, plans, dom_lo, dom_size, tup, seconds=6.0):
    """The same serial bitset CT on every host core: one independent replica
    per thread, each replaying the planned calls with their saves and restores
    (the C calls release the GIL, so the replicas run in parallel)."""
    import threading
    from oracle.serial_ct import SerialCT
    import paper_2507_18413_gb300.ct as C
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    full = C.masks_to_words([np.ones(d, bool) for d in dom_size])
    inputs = [[w.copy() for w in rp.inputs] for rp in plans]
    counts = [0] * cores
    ready = threading.Barrier(cores + 1)
    stop = threading.Event()

    def worker(k):
        ct = SerialCT(dom_lo, dom_size, tup)
        ct.propagate(full.copy())
        ct.save()
        ready.wait()
        done = 0
        while not stop.is_set():
            for rp, ins in zip(plans, inputs):
                buf = [w.copy() for w in ins]
                for op in rp.ops:
                    if op[0] == "save":
                        ct.save()
                    elif op[0] == "restore":
                        ct.restore(op[1])
                    else:
                        ct.propagate(buf[op[1]])
                        done += 1
                if stop.is_set():
                    break
        counts[k] = done
        ct.close()

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(cores)]
    for th in threads:
        th.start()
    ready.wait()
    t0 = time.perf_counter()
    time.sleep(seconds)
    stop.set()
    for th in threads:
        th.join()
    dt = time.perf_counter() - t0
    total = sum(counts)
    return {"value": round(total / dt, 1), "unit": UNIT, "cores": cores,
            "kind": "serial bitset CT (Algorithms 1-3), one independent replica per core",
            "sample": f"{total} propagations of the timed stream with their saves/restores over {cores} threads, "
                      f"{dt:.1f} s"}


def cpu_baseline(args, plans, dom_lo, dom_size, tup):
    from oracle import ct_oracle as O
    import paper_2507_18413_gb300.ct as C
    tup_ret = O.retained_tuples(tup, dom_lo, dom_size)
    inputs = [w for rp in plans for w in rp.inputs]
    done, t0 = 0, time.perf_counter()
    while done < len(inputs) and time.perf_counter() - t0 < args.cpu_seconds:
        O.gac_table(tup_ret, dom_lo, C.words_to_masks(inputs[done], dom_size))
        done += 1
    dt = time.perf_counter() - t0
    return {"value": round(done / dt, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {done} propagations of the timed stream ({args.tuples} tuples), "
                      f"{dt:.1f} s, numpy single thread"}


def run_reference(args, rank, world):
    """The CPU oracle on the same workload: each step a bounded sample of the stream."""
    from oracle import ct_oracle as O
    seed = args.seed
    dom_lo, dom_size, tup = G.large_table(seed, args.tuples, ARITY, DOM)
    tup_ret = O.retained_tuples(tup, dom_lo, dom_size)
    st, root, _ = O.gac_table(tup_ret, dom_lo, [np.ones(d, bool) for d in dom_size])
    per_step = max(1, int(os.environ.get("CT_REF_CALLS", "4")))
    times, props = [], 0
    for s in range(args.warmup + args.steps):
        rng = G.Rng(G.derive_seed(seed, s))
        masks, d = root, 0
        t0 = time.perf_counter()
        for c in range(per_step):
            new = next_edit(rng, masks)
            st, out, _ = O.gac_table(tup_ret, dom_lo, new)
            d += 1
            if st == O.INFEASIBLE or d >= args.depth:
                masks, d = root, 0
            else:
                masks = out
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            props += per_step
    total = sum(times)
    value = props / total
    return {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total * 1e3 / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (seeded SplitMix64)", "impl": "reference",
            "config": {"workload": f"ct_stream_t{args.tuples}_arity{ARITY}_d{DOM}", "tuples": args.tuples,
                       "arity": ARITY, "domain": DOM, "calls_per_step": per_step, "dive_depth": args.depth},
            "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{per_step} propagations of the stream per step, numpy single thread"},
            "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank, world)))
        return
    if args.case != "stream":
        import torch
        from paper_2507_18413_gb300 import build as B
        from paper_2507_18413_gb300 import ct as C
        B.build()
        C.load()
        stream = torch.cuda.current_stream()
        if args.case == "search":
            print(json.dumps(search_extras(C)))
        elif args.case == "planning":
            print(json.dumps(planning_extras(C, n_eval=10)))
        elif args.case == "net512":
            print(json.dumps(network_extras(C)))
        elif args.case == "learned":
            print(json.dumps(learned_extras(C, n_train=200, n_eval=args.learned_eval, node_limit=20_000,
                                            full_eval=args.learned_full)))
        elif args.case == "bulk1e6":
            print(json.dumps(_bulk_update(C, torch, stream, 1_000_000, 6, 32, 5)))
        elif args.case == "stream1e7":
            print(json.dumps(_stream_rate(C, torch, stream, 10_000_000, 128, 99 + 10_000_000, arity=5, d=64,
                                          roofline=True)))
        elif args.case == "bulk4e6":
            print(json.dumps(_bulk_update(C, torch, stream, 4_000_000, 6, 32, 5)))
        else:
            print(json.dumps(_bulk_update(C, torch, stream, 10_000_000, 5, 64, 6)))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    res = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
