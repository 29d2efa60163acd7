#!/usr/bin/env python3
"""Benchmark of the (alpha, beta)-core library on one GB300 (or N replicas under torchrun).

Default workload: the seeded Chung-Lu graph with |U| = 100M, |V| = 50M and 1.5B edges
(exponents 2.0 / 2.3, seed 3). One step is the single (64,64) core, one abcore_compute call on
the resident CSR (the one-time CSR build is timed separately and reported in config). The metric
is peel GTEPS: input edges per second per peel, summed over the queries of a step and over all
ranks. The same line carries the batched form on the same graph (the 8 x 8 log-spaced grid in
[1, 1024], one abcore_compute_batch call, against one plain launch per pair), the roofline of the
dominant kernel, the CPU oracle's time on the host cores, and the oracle parity of (64,64) and of
eight sampled grid pairs.

Other workloads (--workload): "peel-4Mx2M-80M" (five plain peels per step on the 80M-edge
graph), "batch-20Mx10M-500M" / "billion-batch" (batched cores/s), "serve-10Mx5M-200M"
(edge-query latency), "sweep" or "sweep:<graph workload>" (the paper's alpha/beta sensitivity
protocol, GCC against GCC+). --impl reference times the CPU oracle on the same workload.

One JSON line is printed by rank 0.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 256 << 20
PEAK_FALLBACK_GBS = 6800.0


# ------------------------------------------------------------------------------------------
# environment: ranks, peaks, clocks
# ------------------------------------------------------------------------------------------
def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world, backend):
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return PEAK_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed region runs."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id, period_ms=20):
        self.gpu_id = gpu_id
        self.period_ms = period_ms
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", str(self.period_ms), "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.15)

    def stop(self):
        if self.proc is not None:
            time.sleep(0.05)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 10:
                        rows.append(parts)
            os.unlink(self.path)
        except Exception:
            pass
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": len(rows)}
        sm = []
        for r in rows:
            try:
                sm.append(float(r[2]))
                out["sm_max_mhz"] = float(r[3])
            except ValueError:
                pass
            for name, col in (("hw_slowdown", 6), ("hw_thermal_slowdown", 7), ("sw_thermal_slowdown", 8),
                              ("sw_power_cap", 9)):
                if r[col].lower().startswith("active") and name not in out["reasons"]:
                    out["reasons"].append(name)
        if sm:
            out["sm_mhz"] = statistics.median(sm)
        return out


def gpu_uuid(dev):
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev)


# ------------------------------------------------------------------------------------------
# roofline bookkeeping: the survey's per-unit byte figures for a peel (its measurement table):
#   per vertex the scan touches  8 B offsets + 4 B degree (count) write,  1 B mask per vertex,
#   per removed vertex           16 B offsets + 8 B queue write and read,
#   per adjacency entry read     4 B,   per decrement 8 B (a 4-byte read-modify-write),
#   per frontier vertex checked  4 B.
# Each kernel kind is charged those figures for the units its launches processed, from the
# library's counters. Work this design does on top (its row-search sectors beyond the deciding
# entry, the row-prefix lengths, the ticket queue's slot resets and extra row chunks, the
# caller-order gather's id and bitmap reads) is "design overhead": reported apart, never counted
# toward the roofline.
# ------------------------------------------------------------------------------------------
# kernel kinds as the library times them: 1 is the first round (the violator stream, the
# no-return walk of the initial candidate violators, and the scan after them)
KERNEL_NAMES = {0: "k_init", 1: "k_stream+k_round0+k_scan", 2: "k_cascade", 3: "k_batch", 4: "k_serve"}

COUNTER_KEYS = ("peels", "candidates", "init_vertices", "search_probes", "stream_entries", "stream_decrements",
                "scanned", "round0_rows", "entries", "decrements", "pushes", "items", "emit_gathered",
                "emit_scattered", "mask_zeroed", "hub_decrements", "hub_flushes")


def algorithmic_bytes(st):
    """(algorithmic bytes, design overhead bytes) per kernel kind, from accumulated counters."""
    alg, over = {}, {}
    # count init: a candidate's offsets and count; a row-search probe decides on one entry
    alg[0] = 12 * st["init_vertices"] + 4 * st["search_probes"]
    over[0] = 4 * st["init_vertices"] + 28 * st["search_probes"]  # row prefix; rest of each sector
    # first round: streamed entries and their decrements, the candidates checked after them, and
    # the rows walked for the initial candidate violators (offsets and queue entry each)
    r0 = st.get("round0_rows", 0)
    alg[1] = 4 * st["stream_entries"] + 8 * st["stream_decrements"] + 4 * st.get("scanned", 0) + 24 * r0
    over[1] = 8 * r0  # a round0 list entry is 16 B written and read, against 8 B of queue
    # cascade: every vertex the queue carried, its entries and decrements, and the masks
    removed = max(st["pushes"] - r0, 0)
    dec_casc = st["decrements"] - st["stream_decrements"]
    alg[2] = 24 * removed + 4 * st["entries"] + 8 * dec_casc + st["emit_gathered"] + st.get("mask_zeroed", 0)
    # the queue moves 36 B per item (slot write, read and reset, offset, row length) against 24 B
    # per removed vertex; the gather reads 4 B of caller-order id and 1/4 B of bitmap per vertex,
    # and each removal sets its bit (8 B); the scatter reads 4 B of count per candidate, and its
    # survivor bitmap is read and cleared by the expansion (1/4 B per vertex)
    over[2] = (max(36 * st["items"] - 24 * removed, 0)
               + (4.25 * st["emit_gathered"] + 8 * removed if st["emit_gathered"] > 0 else 0)
               + 4 * st["emit_scattered"] + st.get("mask_zeroed", 0) / 4)
    return alg, over


def cpu_info():
    """CPU model and logical core count of this host (lscpu when present)."""
    model, vendor, ncpu = None, None, os.cpu_count()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() == "Model name" and model is None:
                model = v.strip()
            elif k.strip() == "Vendor ID" and vendor is None:
                vendor = v.strip()
    except Exception:
        pass
    if model and vendor and vendor not in model:
        model = "%s %s" % (vendor, model)
    model = model or vendor
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"cpu_model": model, "host_cores": ncpu}


def oracle_threads():
    """Oracle runs done side by side in host threads (each one single-threaded)."""
    import oracle
    return oracle.default_threads()


def oracle_peels(nU, nV, off, adj, pairs, threads=None):
    """{pair: (mask_u, mask_v, seconds)} of the oracle, several pairs peeled at once."""
    import oracle
    return oracle.peel_many(nU, nV, off, adj, pairs, threads)


def source_digest():
    """Digest of the peel and batch kernels' sources with // comments and blank lines dropped, so
    that only a change of code (not of its commentary) retires a recorded ncu figure."""
    h = hashlib.sha256()
    for fn in ("peel.cu", "batch.cu", "peel_core.cuh", "device.cuh", "internal.h"):
        with open(os.path.join(ROOT, "paper_2606_07148_gb300", "csrc", fn)) as f:
            for line in f:
                code = line.split("//", 1)[0].strip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def traffic_from_profiles(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is unchanged."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(p):
        return None
    dig = source_digest()
    with open(p) as f:
        for line in f:
            t = line.split()
            if len(t) >= 4 and not line.startswith("#") and t[0] == kernel and t[1] == workload:
                return float(t[2]) if t[3] == dig else None
    return None


# ------------------------------------------------------------------------------------------
# workloads
# ------------------------------------------------------------------------------------------
def make_inputs(name, device):
    import synth
    spec = synth.WORKLOADS[name]
    nU, nV, eu, ev = synth.make_graph(spec, device=device)
    return spec, nU, nV, eu, ev


def describe(spec, name):
    return ("Chung-Lu bipartite |U|=%d |V|=%d m=%d exponents %.1f/%.1f seed %d"
            % (spec["nU"], spec["nV"], spec["m"], spec["gamma_u"], spec["gamma_v"], spec["seed"]))


def peel_pairs_for(name, spec):
    if name.startswith("billion"):
        return [tuple(spec["pairs"][0])]
    return [tuple(p) for p in spec["pairs"]]


def grid_pairs_for(name, spec):
    """The grid batched beside the single peel: the 8 x 8 grid on the 1.5B-edge graph."""
    if name.startswith("billion"):
        return [tuple(p) for p in spec["pairs"][1:]]
    return []


def sampled_grid_pairs(grid, limit):
    import synth
    return synth.sampled_pairs(grid, limit)


def cpu_baseline_peel(nU, nV, off, adj, pairs, m, budget_s=25.0):
    """The oracle as it stands, single-threaded, on the step's queries in turn until the budget is
    spent (at least one query). Returns the baseline record and the masks it computed."""
    import oracle
    done = 0
    t0 = time.perf_counter()
    results = {}
    for a, b in pairs:
        results[(a, b)] = oracle.peel(nU, nV, off, adj, a, b)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    rec = {"value": done * m / dt / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
           "sample": "%d of the %d queries of one step (%s), single-threaded oracle peel, CSR build excluded"
                     % (done, len(pairs), ", ".join("(%d,%d)" % p for p in list(results)))}
    rec.update(cpu_info())
    return rec, results


def batch_leg(core, args, dev, nU, nV, grid, flush, timed_steps):
    """The grid as one abcore_compute_batch call (a CUDA-graph replay), against one plain
    abcore_compute launch per pair on the same GPU. Returns (record, device masks)."""
    import torch
    a = [p[0] for p in grid]
    b = [p[1] for p in grid]
    tuned, tune_s = None, 0.0
    peel_params = {k: core.get_param(k) for k in core.TUNED}
    if not args.no_autotune:
        t = time.perf_counter()
        _, tuned = core.autotune(grid, batch=True)
        tune_s = time.perf_counter() - t
        apply_params(core, args)
    mu = torch.empty((len(grid), nU), dtype=torch.uint8, device=dev)
    mv = torch.empty((len(grid), nV), dtype=torch.uint8, device=dev)
    for _ in range(max(args.warmup, 1)):
        core.compute_batch(a, b, mu, mv)
    core.set_param("timing", 1)
    core.set_param("reset_stats", 1)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(timed_steps)]
    torch.cuda.synchronize()
    for i in range(timed_steps):
        flush.fill_(i & 0xFF)
        evs[i][0].record()
        core.compute_batch(a, b, mu, mv)
        evs[i][1].record()
    torch.cuda.synchronize()
    st = core.stats()
    core.set_param("timing", 0)
    launches = st["launches"]  # counted since the reset: the timed calls only
    ms = statistics.mean([x.elapsed_time(y) for x, y in evs])
    alg, over = algorithmic_bytes(st)
    kb, ko = alg[0] + alg[1] + alg[2], over[0] + over[1] + over[2]
    kms, nl = st["kernel_ms"][3], max(st["kernel_launches"][3], 1)
    peak, peak_src = measured_peaks()
    achieved = kb / nl / (kms / nl / 1e3) / 1e9 if kms > 0 else 0.0
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "kernel": "k_batch+k_batch_emit", "peak_source": peak_src,
                "algorithmic_bytes_per_launch": int(kb / nl), "design_overhead_bytes_per_launch": int(ko / nl),
                "avg_launch_ms": round(kms / nl, 3)}
    counters = {k: round(st[k] / nl) for k in COUNTER_KEYS}
    # comparator: one plain (GCC) launch per pair with the single peel's own parameters, every
    # pair also checked against the batch
    for k, v in peel_params.items():
        core.set_param(k, v)
    apply_params(core, args)
    algo = core.get_param("algo")
    core.set_param("algo", 1)
    ou = torch.empty(nU, dtype=torch.uint8, device=dev)
    ov = torch.empty(nV, dtype=torch.uint8, device=dev)
    for x, y in grid[:4]:
        core.compute(x, y, ou, ov)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.fill_(7)
    c0.record()
    for x, y in grid:
        core.compute(x, y, ou, ov, asynchronous=True)
    c1.record()
    core.sync()
    torch.cuda.synchronize()
    plain_ms = c0.elapsed_time(c1)
    mism = 0
    for i, (x, y) in enumerate(grid):
        core.compute(x, y, ou, ov)
        mism += int(not (torch.equal(ou, mu[i]) and torch.equal(ov, mv[i])))
    core.set_param("algo", algo)
    rec = {"metric": "batched (alpha,beta)-cores/s", "value": round(len(grid) / (ms / 1e3), 2), "unit": "cores/s",
           "pairs": len(grid), "grid": sorted(set(a)), "ms_per_batch": round(ms, 3), "steps": timed_steps,
           "roofline": roofline, "counters_per_batch": counters,
           "plain_one_launch_per_pair": {"ms": round(plain_ms, 3),
                                         "cores_per_s": round(len(grid) / (plain_ms / 1e3), 2),
                                         "batch_speedup": round(plain_ms / ms, 2)},
           "batch_equals_plain_pairs": "%d/%d" % (len(grid) - mism, len(grid)),
           "autotuned": tuned, "autotune_s": round(tune_s, 2), "gpu_launches": launches}
    return rec, (mu, mv)


def run_peel(args, rank, world, local):
    import numpy as np
    import torch
    from paper_2606_07148_gb300 import ABCore

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    name = args.workload
    spec, nU, nV, eu, ev = make_inputs(name, dev)
    m = spec["m"]
    pairs = peel_pairs_for(name, spec)
    grid = grid_pairs_for(name, spec) if not args.no_batch else []
    core = ABCore(local)
    core.set_param("algo", 1)  # the headline is the plain (index-free) peel; GCC+ is reported apart
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    core.load_edges(nU, nV, eu, ev)
    e1.record()
    torch.cuda.synchronize()
    csr_ms = e0.elapsed_time(e1)
    tuned, tune_s = None, 0.0
    apply_params(core, args)  # (untuned settings apply to the tuning runs too)
    if not args.no_autotune:
        t = time.perf_counter()
        _, tuned = core.autotune(pairs)
        tune_s = time.perf_counter() - t
    apply_params(core, args)
    want_oracle = rank == 0 and world == 1 and not args.no_cpu_baseline
    eu_h = eu.cpu().numpy() if want_oracle else None
    ev_h = ev.cpu().numpy() if want_oracle else None
    del eu, ev
    torch.cuda.empty_cache()

    outs = [(torch.empty(nU, dtype=torch.uint8, device=dev), torch.empty(nV, dtype=torch.uint8, device=dev))
            for _ in pairs]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step():
        for (a, b), (ou, ov) in zip(pairs, outs):
            core.compute(a, b, ou, ov, asynchronous=True)

    # warm-up; its last step is instrumented with CUDA events around every kernel kind, which
    # gives the kernel shares and picks the dominant kind
    n_warm = max(args.warmup, 1)
    for i in range(n_warm):
        if i == n_warm - 1:
            core.set_param("timing", 1)
            core.set_param("timing_kinds", 0xFF)
            core.set_param("reset_stats", 1)
        flush.fill_(1)
        step()
    core.sync()
    stw = core.stats()
    warm_ms = stw["kernel_ms"]
    dom = max((k for k in (0, 1, 2)), key=lambda k: warm_ms[k])
    # the timed steps record events around the dominant kind's launches only: an event between
    # two kernels costs the step about as much as a launch (every kind timed: ~7 % slower)
    core.set_param("timing_kinds", 1 << dom)
    core.set_param("reset_stats", 1)
    st0 = core.stats()
    clocks = ClockSampler(gpu_uuid(local))
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        evs[i][0].record()
        step()
        evs[i][1].record()
    core.sync()
    torch.cuda.synchronize()
    barrier(world)
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    st = core.stats()
    core.set_param("timing", 0)
    core.set_param("timing_kinds", 0xFF)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = statistics.mean(step_ms)
    ms = allreduce_max(ms, world, dev)
    value = world * len(pairs) * m / (ms / 1e3) / 1e9

    launches = st["launches"] - st0["launches"]
    alg, over = algorithmic_bytes(st)
    kern_ms = st["kernel_ms"]
    n_launch = max(st["kernel_launches"][dom], 1)
    achieved = alg[dom] / n_launch / (kern_ms[dom] / n_launch / 1e3) / 1e9 if kern_ms[dom] > 0 else 0.0
    peak, peak_src = measured_peaks()
    traffic = traffic_from_profiles(KERNEL_NAMES[dom], name)
    steps = max(args.steps, 1)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "kernel": KERNEL_NAMES[dom], "peak_source": peak_src,
                "algorithmic_bytes_per_launch": int(alg[dom] / n_launch),
                "design_overhead_bytes_per_launch": int(over[dom] / n_launch),
                "avg_launch_ms": round(kern_ms[dom] / n_launch, 4),
                "timed": "CUDA events around this kind's launches in every timed step",
                "kernel_share": {KERNEL_NAMES[k]: round(warm_ms[k] / max(sum(warm_ms[:3]), 1e-9), 3)
                                 for k in (0, 1, 2)},
                "kernel_share_from": "the last warm-up step, every kind timed",
                "counters_per_step": {k: round(st[k] / steps) for k in COUNTER_KEYS},
                "bytes_per_step": {KERNEL_NAMES[k]: {"algorithmic": int(alg[k] / steps),
                                                     "design_overhead": int(over[k] / steps)} for k in (0, 1, 2)}}

    # the ceiling that binds a peel whose counts sit in L2: the device's rate of random 4-byte
    # atomics, with the old value returned (the cascade's crossing test) and without (the first
    # round's decrements); the library measures both (the kind's time from the timed steps when
    # it is the dominant kind, else from the instrumented warm-up step)
    at_ret, at_noret = core.measure_atomics(32 << 20)

    def rate(kind, decs):
        sa, kms = (st, kern_ms[kind]) if dom == kind else (stw, warm_ms[kind])
        return decs(sa) / (kms / 1e3) if kms > 0 else 0.0
    casc = rate(2, lambda x: x["decrements"] - x["stream_decrements"])
    first = rate(1, lambda x: x["stream_decrements"])
    # decrements summed in a block's shared-memory hub table reach L2 as one atomic per table entry
    first_l2 = rate(1, lambda x: x["stream_decrements"] - x["hub_decrements"] + x["hub_flushes"])
    l2_atomics = {"unit": "G/s",
                  "k_cascade": {"decrements_per_s": round(casc / 1e9, 2), "peak_per_s": round(at_ret / 1e9, 2),
                                "frac": round(casc / at_ret, 4) if at_ret > 0 else None, "returns": True},
                  "k_stream+k_round0+k_scan": {"decrements_per_s": round(first / 1e9, 2),
                                               "l2_atomics_per_s": round(first_l2 / 1e9, 2),
                                               "peak_per_s": round(at_noret / 1e9, 2),
                                               "frac": round(first / at_noret, 4) if at_noret > 0 else None,
                                               "l2_frac": round(first_l2 / at_noret, 4) if at_noret > 0 else None,
                                               "returns": False},
                  "probe": "2^26 random atomicSub over a 32 MB int array (L2-resident), abcore_measure_atomics"}

    # end to end through the C ABI with host buffers (pinned): per step, the queries' thresholds
    # go in as call arguments and every mask comes back to the host inside the timed region
    host = [(torch.empty(nU, dtype=torch.uint8, pin_memory=True), torch.empty(nV, dtype=torch.uint8, pin_memory=True))
            for _ in pairs]
    e2e_steps = max(1, min(args.steps, 50))
    for (a, b), (hu, hv) in zip(pairs, host):
        core.compute(a, b, hu, hv)
    barrier(world)
    t = time.perf_counter()
    for _ in range(e2e_steps):
        for (a, b), (hu, hv) in zip(pairs, host):
            core.compute(a, b, hu, hv)
    e2e_s = (time.perf_counter() - t) / e2e_steps
    e2e_s = allreduce_max(e2e_s, world, dev)
    e2e = {"value": round(world * len(pairs) * m / e2e_s / 1e9, 3), "unit": "GTEPS",
           "h2d_bytes_per_step": 8 * len(pairs), "d2h_bytes_per_step": len(pairs) * (nU + nV)}

    # Algorithm 2 (GCC+): one-time core decomposition and core-ordered layout, then the same
    # queries pruned by Lemma 1 (each query takes whichever of GCC / GCC+ leaves fewer vertices)
    gccp = None
    if not args.no_gccplus:
        torch.cuda.synchronize()
        t = time.perf_counter()
        _, _, maxcore = core.core_numbers()
        torch.cuda.synchronize()
        prep_ms = (time.perf_counter() - t) * 1e3
        core.set_param("algo", 0)
        ref = [(ou.clone(), ov.clone()) for ou, ov in outs]
        for _ in range(args.warmup):
            flush.fill_(1)
            step()
        core.sync()
        pevs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            pevs[i][0].record()
            step()
            pevs[i][1].record()
        core.sync()
        torch.cuda.synchronize()
        pms = allreduce_max(statistics.mean([a.elapsed_time(b) for a, b in pevs]), world, dev)
        same = all(torch.equal(r[0], o[0]) and torch.equal(r[1], o[1]) for r, o in zip(ref, outs))
        del ref
        # the paper's default query (Section 6), computed by the library
        delta, qa, qoff, qb = core.default_query()

        def one(algo):
            core.set_param("algo", algo)
            ou, ov = outs[0]
            core.compute(qa, qb, ou, ov)
            best = 1e9
            for i in range(5):
                flush.fill_(i)
                x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                x0.record()
                core.compute(qa, qb, ou, ov, asynchronous=True)
                x1.record()
                core.sync()
                torch.cuda.synchronize()
                best = min(best, x0.elapsed_time(x1))
            return round(best, 4)

        default_q = {"delta": delta, "alpha": qa, "alpha_offset": qoff, "beta": qb,
                     "gcc_ms": one(1), "gccplus_ms": one(2)}
        gccp = {"preprocess_ms": round(prep_ms, 2), "max_core": maxcore, "ms_per_step": round(pms, 4),
                "value": round(world * len(pairs) * m / (pms / 1e3) / 1e9, 3), "unit": "GTEPS",
                "masks_identical_to_plain": same, "paper_default_query": default_q,
                "note": "per query the pruned peel runs when it leaves fewer vertices than the plain one; "
                        "preprocessing (core decomposition + core-ordered CSR) is excluded from ms_per_step"}
        core.set_param("algo", 1)

    batch, bmasks = None, None
    if grid:
        batch, bmasks = batch_leg(core, args, dev, nU, nV, grid, flush, max(1, min(args.steps, 10)))

    cpu = None
    parity = None
    if eu_h is not None:
        import oracle
        t = time.perf_counter()
        off, adj = oracle.build_csr(nU, nV, eu_h, ev_h)
        del eu_h, ev_h
        csr_s = time.perf_counter() - t
        cpu, res = cpu_baseline_peel(nU, nV, off, adj, pairs, m)
        cpu["oracle_csr_build_s"] = round(csr_s, 1)
        ok = 0
        for (a, b), (hu, hv) in zip(pairs, host):
            if (a, b) in res:
                wu, wv = res[(a, b)]
                ok += int(np.array_equal(hu.numpy(), wu) and np.array_equal(hv.numpy(), wv))
        parity = {"single": "%d/%d queries bit-exact vs oracle (%s)"
                            % (ok, len(res), ", ".join("(%d,%d)" % p for p in res))}
        if grid:
            sample = sampled_grid_pairs(grid, 8)
            t = time.perf_counter()
            om = oracle_peels(nU, nV, off, adj, sample)
            okb = 0
            for p in sample:
                i = grid.index(p)
                wu, wv, _ = om[p]
                okb += int(np.array_equal(bmasks[0][i].cpu().numpy(), wu) and np.array_equal(bmasks[1][i].cpu().numpy(), wv))
            parity["batch"] = ("%d/%d sampled grid pairs bit-exact vs oracle (%s); every pair equal to its plain "
                               "peel: %s" % (okb, len(sample), ", ".join("(%d,%d)" % p for p in sample),
                                             batch["batch_equals_plain_pairs"]))
            parity["oracle_threads"] = oracle_threads()
            parity["oracle_wall_s"] = round(time.perf_counter() - t, 1)
        del off, adj

    line = {
        "metric": "(alpha,beta)-core peel GTEPS", "value": round(value, 3), "unit": "GTEPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": name, "graph": describe(spec, name), "queries_per_step": [list(p) for p in pairs],
                   "csr_build_ms": round(csr_ms, 2), "parallelism": "replicas" if world > 1 else "single",
                   "l2": "flushed before every step (256 MB write); CSR %.2f GB > 129 MB L2"
                         % ((8 * (nU + nV + 1) + 8 * m) / 1e9),
                   "timed_wall_s": round(t_wall, 4), "algorithm": "GCC (plain peel, Algorithm 1)",
                   "autotuned": tuned, "autotune_s": round(tune_s, 2), "params": args.param},
        "clocks": clk, "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "l2_atomics": l2_atomics,
        "cpu_baseline": cpu, "parity": parity, "gccplus": gccp, "batch": batch,
        "step_ms": {"min": round(min(step_ms), 4), "median": round(statistics.median(step_ms), 4)},
    }
    core.close()
    return line


def run_batch(args, rank, world, local):
    """Batched cores/s: all pairs of the grid in one abcore_compute_batch call (a graph replay)."""
    import numpy as np
    import torch
    from paper_2606_07148_gb300 import ABCore

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    base = "billion-100Mx50M-1500M" if args.workload == "billion-batch" else args.workload
    spec, nU, nV, eu, ev = make_inputs(base, dev)
    pairs = [tuple(p) for p in spec["pairs"]]
    if base.startswith("billion"):
        pairs = pairs[1:]  # the 8 x 8 grid; the single (64, 64) core is the peel workload
    core = ABCore(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    core.load_edges(nU, nV, eu, ev)
    e1.record()
    torch.cuda.synchronize()
    csr_ms = e0.elapsed_time(e1)
    want_oracle = rank == 0 and world == 1 and not args.no_cpu_baseline
    eu_h = eu.cpu().numpy() if want_oracle else None
    ev_h = ev.cpu().numpy() if want_oracle else None
    del eu, ev
    torch.cuda.empty_cache()
    apply_params(core, args)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    steps = max(1, args.steps)
    clocks = ClockSampler(gpu_uuid(local))
    clocks.start()
    barrier(world)
    t_wall0 = time.perf_counter()
    rec, (mu, mv) = batch_leg(core, args, dev, nU, nV, pairs, flush, steps)
    barrier(world)
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    ms = allreduce_max(rec["ms_per_batch"], world, dev)
    value = world * len(pairs) / (ms / 1e3)
    # end to end with host buffers: every mask of every pair comes back each step
    a = [p[0] for p in pairs]
    b = [p[1] for p in pairs]
    e2e = None
    if len(pairs) * (nU + nV) <= (8 << 30):
        hu = torch.empty((len(pairs), nU), dtype=torch.uint8, pin_memory=True)
        hv = torch.empty((len(pairs), nV), dtype=torch.uint8, pin_memory=True)
        core.compute_batch(a, b, hu, hv)
        e2e_steps = max(1, min(steps, 3))
        t = time.perf_counter()
        for _ in range(e2e_steps):
            core.compute_batch(a, b, hu, hv)
        e2e_s = allreduce_max((time.perf_counter() - t) / e2e_steps, world, dev)
        e2e = {"value": round(world * len(pairs) / e2e_s, 2), "unit": "cores/s", "h2d_bytes_per_step": 8 * len(pairs),
               "d2h_bytes_per_step": len(pairs) * (nU + nV)}
        del hu, hv
    cpu, parity = None, None
    if eu_h is not None:
        import oracle
        t = time.perf_counter()
        off, adj = oracle.build_csr(nU, nV, eu_h, ev_h)
        del eu_h, ev_h
        csr_s = time.perf_counter() - t
        n_alpha = len({p[0] for p in pairs})
        sample = sampled_grid_pairs(pairs, 2 * n_alpha + 4)
        t = time.perf_counter()
        om = oracle_peels(nU, nV, off, adj, sample)
        wall = time.perf_counter() - t
        ok = 0
        for p in sample:
            i = pairs.index(p)
            wu, wv, _ = om[p]
            ok += int(np.array_equal(mu[i].cpu().numpy(), wu) and np.array_equal(mv[i].cpu().numpy(), wv))
        parity = ("%d/%d sampled pairs bit-exact vs oracle (grid corners, then every chain's first and last beta); "
                  "every pair equal to its plain peel: %s" % (ok, len(sample), rec["batch_equals_plain_pairs"]))
        secs = sum(v[2] for v in om.values())
        cpu = {"value": round(len(sample) / secs, 4), "unit": "cores/s", "cores": 1, "kind": "oracle",
               "sample": "%d grid pairs, each a single-threaded oracle peel (%d run side by side, %.1f s wall); "
                         "value = pairs / summed per-pair seconds; CSR build (%.1f s) excluded"
                         % (len(sample), oracle_threads(), wall, csr_s)}
        cpu.update(cpu_info())
        del off, adj
    rec["roofline"]["traffic"] = traffic_from_profiles("k_batch", args.workload)
    line = {
        "metric": "batched (alpha,beta)-cores/s", "value": round(value, 2), "unit": "cores/s",
        "n_gpus": world, "steps": steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "graph": describe(spec, base), "pairs": len(pairs),
                   "grid": sorted(set(a)), "csr_build_ms": round(csr_ms, 2),
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "flushed before every step (256 MB write)", "timed_wall_s": round(t_wall, 3),
                   "params": args.param, "autotuned": rec["autotuned"], "autotune_s": rec["autotune_s"]},
        "clocks": clk, "e2e": e2e, "gpu_launches": rec["gpu_launches"], "roofline": rec["roofline"],
        "counters_per_batch": rec["counters_per_batch"],
        "plain_one_launch_per_pair": rec["plain_one_launch_per_pair"],
        "cpu_baseline": cpu, "parity": parity,
    }
    core.close()
    return line


def stream_sample_positions(stream, n_targets, per):
    import synth
    return synth.sample_positions(stream, n_targets, per)


def run_serve(args, rank, world, local):
    """Edge-query serving: the update stream replayed open-loop at each arrival rate."""
    import numpy as np
    import torch
    import synth
    from paper_2606_07148_gb300 import ABCore, abi

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    spec, nU, nV, eu, ev = make_inputs(args.workload, dev)
    m = spec["m"]
    eu_h, ev_h = eu.cpu().numpy(), ev.cpu().numpy()
    n_ops = args.serve_ops or spec["n_ops"]
    t0 = time.perf_counter()
    stream = synth.edge_update_stream(eu_h, ev_h, nU, nV, n_ops, spec["seed"])
    gen_s = time.perf_counter() - t0
    targets = [tuple(t) for t in spec["targets"]]
    reqs = (abi.abcore_req * n_ops)()
    for k in range(n_ops):
        reqs[k].op = int(stream.op[k]); reqs[k].u = int(stream.u[k]); reqs[k].v = int(stream.v[k])
        reqs[k].target = int(stream.target[k]); reqs[k].tag = k
    req_size = ctypes_sizeof(abi.abcore_req)
    results = {}
    answers = {}
    # the host loop must not stall: responses land in one reused numpy buffer (no Python object
    # per response), the collector is paused, and the clock sampler polls every 100 ms (its power
    # and throttle queries, at 20 ms, were seen to hold the serving loop up for ~30 ms at a time)
    clocks = ClockSampler(gpu_uuid(local), period_ms=100)
    clocks.start()
    buf = np.zeros(8192, dtype=ABCore.RESP_DTYPE)
    import gc
    for rate in spec["rates"]:
        core = ABCore(local)
        core.load_edges(nU, nV, eu, ev)
        core.serve_start(targets, ring_slots=8192)
        sched = stream.t_unit / rate
        done_t = np.zeros(n_ops)
        in_core = np.zeros(n_ops, dtype=np.uint8)
        got = 0
        k = 0
        gc.collect()
        gc.disable()
        start = time.perf_counter()
        while got < n_ops:
            now = time.perf_counter() - start
            if now > sched[-1] + 120.0:
                raise RuntimeError("serving stalled: %d of %d answered" % (got, n_ops))
            hi = int(np.searchsorted(sched, now, side="right"))
            hi = min(hi, k + 4096)
            if hi > k:
                sub = (abi.abcore_req * (hi - k)).from_buffer(reqs, k * req_size)
                if core.serve_submit(sub) is not None:
                    k = hi
            out = core.serve_poll_into(buf)
            if len(out):
                tnow = time.perf_counter() - start
                seqs = out["seq"].astype(np.int64)
                done_t[seqs] = tnow
                in_core[seqs] = out["in_core"]
                got += len(out)
        gc.enable()
        core.serve_stop()
        sst = core.stats()
        lat_ms = (done_t - sched) * 1e3
        elapsed = done_t.max()
        results[str(rate)] = {"p50_ms": round(float(np.percentile(lat_ms, 50)), 4),
                              "p99_ms": round(float(np.percentile(lat_ms, 99)), 4),
                              "max_ms": round(float(lat_ms.max()), 4),
                              "achieved_ops_per_s": round(n_ops / elapsed, 1),
                              "re_peel": {"regions": sst["serve_regions"],
                                          "region_vertices_per_region": round(sst["serve_region_vertices"] / max(sst["serve_regions"], 1), 2),
                                          "cascades": sst["serve_cascades"],
                                          "vertices_per_cascade": round(sst["serve_cascade_vertices"] / max(sst["serve_cascades"], 1), 2)}}
        answers[rate] = in_core.tolist()
        core.close()
    clk = clocks.stop()
    same = all(answers[r] == answers[spec["rates"][0]] for r in spec["rates"])
    cpu, parity = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        off, adj = oracle.build_csr(nU, nV, eu_h, ev_h)
        # baseline: the oracle re-peels the whole graph for a query (on this graph one component
        # holds almost every vertex, so that is also the paper's component-scoped re-peel)
        t = time.perf_counter()
        for tg in targets:
            oracle.peel(nU, nV, off, adj, tg[0], tg[1])
        per_q = (time.perf_counter() - t) / len(targets)
        del off, adj
        cpu = {"value": round(1.0 / per_q, 4), "unit": "queries/s", "cores": 1, "kind": "oracle",
               "sample": "one full single-threaded oracle peel of the base graph per target (%d peels)" % len(targets)}
        cpu.update(cpu_info())
        ks = stream_sample_positions(stream, len(targets), 6)
        ta = np.array([t_[0] for t_ in targets], dtype=np.int32)[stream.target.astype(np.int64)]
        tb = np.array([t_[1] for t_ in targets], dtype=np.int32)[stream.target.astype(np.int64)]
        t = time.perf_counter()
        res = oracle.replay_at(nU, nV, eu_h, ev_h, stream.op, stream.u, stream.v, ta, tb, ks)
        last = answers[spec["rates"][-1]]
        ok = sum(int(res[k][0] == last[k]) for k in ks)
        parity = ("%d/%d sampled updates (both kinds, every target, spread over the stream) answer as the oracle's "
                  "replay of the stream up to them (%.0f s, %d threads); answers identical across rates: %s"
                  % (ok, len(ks), time.perf_counter() - t, oracle_threads(), same))
    # the paper's GFQ scope as an ablation: the first updates of the same stream, each answered by
    # re-peeling the endpoints' components from scratch (query_scope = 1), one call at a time
    n_scope = min(n_ops, args.scope_ops)
    scope = None
    if n_scope > 0:
        core = ABCore(local)
        core.load_edges(nU, nV, eu, ev)
        core.set_param("query_scope", 1)
        lat, got = [], []
        for k in range(n_scope):
            tg = targets[int(stream.target[k])]
            t = time.perf_counter()
            got.append(core.query_edge(int(stream.u[k]), int(stream.v[k]), int(stream.op[k]), tg[0], tg[1]))
            lat.append((time.perf_counter() - t) * 1e3)
        st = core.stats()
        core.close()
        first = answers[spec["rates"][0]]
        scope = {"updates": n_scope, "p50_ms": round(float(np.percentile(lat, 50)), 3),
                 "p99_ms": round(float(np.percentile(lat, 99)), 3), "mean_ms": round(float(np.mean(lat)), 3),
                 "queries_per_s": round(n_scope / (sum(lat) / 1e3), 1),
                 "vertices_repeeled_per_query": round(st["scope_vertices"] / max(st["scope_queries"], 1)),
                 "answers_identical_to_certificate_scope": got == list(first[:n_scope]),
                 "note": "one abcore_query_edge call per update, closed loop (latency is the call's wall time)"}
    # component labels (the GFQ preprocessing) on the base graph, timed on the device
    core = ABCore(local)
    core.load_edges(nU, nV, eu, ev)
    lu = torch.empty(nU, dtype=torch.int32, device=dev)
    lv = torch.empty(nV, dtype=torch.int32, device=dev)
    core.components(lu, lv)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record()
    _, _, ncomp = core.components(lu, lv)
    c1.record()
    torch.cuda.synchronize()
    largest = int(torch.bincount(torch.cat([lu, lv]).long()).max().item())
    comps = {"ms": round(c0.elapsed_time(c1), 3), "components": ncomp, "largest": largest,
             "vertices": nU + nV}
    core.close()
    # comparator on the same GPU: one full plain peel of the graph per query
    core = ABCore(local)
    core.load_edges(nU, nV, eu, ev)
    ou = torch.empty(nU, dtype=torch.uint8, device=dev)
    ov = torch.empty(nV, dtype=torch.uint8, device=dev)
    for tg in targets:
        core.compute(tg[0], tg[1], ou, ov)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record()
    for i in range(40):
        tg = targets[int(stream.target[i])]
        core.compute(tg[0], tg[1], ou, ov, asynchronous=True)
    c1.record()
    core.sync()
    torch.cuda.synchronize()
    plain_qps = 40 / (c0.elapsed_time(c1) / 1e3)
    core.close()
    top = results[str(max(spec["rates"]))]
    line = {
        "metric": "edge-query p99 latency at the highest arrival rate", "value": top["p99_ms"], "unit": "ms",
        "n_gpus": world, "steps": len(spec["rates"]), "warmup": 0, "ms_per_step": None,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "graph": describe(spec, args.workload), "updates": n_ops,
                   "targets": [list(t) for t in targets], "stream_gen_s": round(gen_s, 2),
                   "parallelism": "single"},
        "rates": results, "answers_identical_across_rates": same, "parity": parity, "cpu_baseline": cpu,
        "component_scope": scope,
        "components": comps,
        "plain_full_peel_per_query_qps": round(plain_qps, 1), "clocks": clk,
        "e2e": {"value": top["p99_ms"], "unit": "ms", "h2d_bytes_per_step": n_ops * req_size,
                "d2h_bytes_per_step": n_ops * ctypes_sizeof(abi.abcore_resp)},
    }
    return line


def run_sweep(args, rank, world, local):
    """The paper's alpha/beta sensitivity protocol (Section 6): delta = the largest core number;
    fix beta = 0.5 delta and vary alpha = c delta, then fix alpha = 0.5 delta and vary
    beta = c delta, c = 0.1 .. 0.9; each query timed with the plain peel (GCC) and with the
    core-number pruning (GCC+), L2 flushed before each run."""
    import torch
    from paper_2606_07148_gb300 import ABCore

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    base = args.workload.split(":", 1)[1] if ":" in args.workload else "peel-4Mx2M-80M"
    spec, nU, nV, eu, ev = make_inputs(base, dev)
    m = spec["m"]
    core = ABCore(local)
    core.load_edges(nU, nV, eu, ev)
    del eu, ev
    torch.cuda.synchronize()
    t = time.perf_counter()
    _, _, delta = core.core_numbers()
    torch.cuda.synchronize()
    prep_ms = (time.perf_counter() - t) * 1e3
    ou = torch.empty(nU, dtype=torch.uint8, device=dev)
    ov = torch.empty(nV, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def timed(a, b, algo):
        core.set_param("algo", algo)
        core.compute(a, b, ou, ov)
        best = 1e9
        for i in range(max(args.steps, 1)):
            flush.fill_(i & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            core.compute(a, b, ou, ov, asynchronous=True)
            e1.record()
            core.sync()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return round(best, 4)

    cs = [round(0.1 * i, 1) for i in range(1, 10)]
    half = max(1, int(0.5 * delta))
    rows = []
    for fixed in ("beta", "alpha"):
        for c in cs:
            v = max(1, int(c * delta))
            a, b = (v, half) if fixed == "beta" else (half, v)
            g1, g2 = timed(a, b, 1), timed(a, b, 2)
            rows.append({"vary": "alpha" if fixed == "beta" else "beta", "c": c, "alpha": a, "beta": b,
                         "gcc_ms": g1, "gccplus_ms": g2})
    clk = {"note": "not sampled for the sweep"}
    total_gcc = sum(r["gcc_ms"] for r in rows)
    line = {
        "metric": "alpha/beta sweep: queries/s, plain peel", "value": round(len(rows) / (total_gcc / 1e3), 2),
        "unit": "queries/s", "n_gpus": world, "steps": args.steps, "warmup": 1, "ms_per_step": round(total_gcc, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": "sweep:" + base, "graph": describe(spec, base), "delta": delta,
                   "core_numbers_ms": round(prep_ms, 2), "edges": m,
                   "l2": "flushed before every timed query (256 MB write)"},
        "gccplus_queries_per_s": round(len(rows) / (sum(r["gccplus_ms"] for r in rows) / 1e3), 2),
        "queries": rows, "clocks": clk,
    }
    core.close()
    return line


def apply_params(core, args):
    for kv in args.param:
        k, v = kv.split("=", 1)
        core.set_param(k, int(v))


def ctypes_sizeof(t):
    import ctypes
    return ctypes.sizeof(t)


def run_reference(args, rank, world, local):
    """The CPU oracle on the same workload, metric and config. A step is one oracle peel of the
    step's queries in turn (rotating); the peels of the timed steps run side by side in host
    threads, each one the plain single-threaded oracle, so the run ends within minutes even on
    the 1.5B-edge graph (about 20 s per peel there)."""
    import concurrent.futures as cf
    import torch
    import oracle
    import synth
    if rank != 0:
        return None
    name = args.workload
    spec = synth.WORKLOADS[name]
    device = "cuda" if torch.cuda.is_available() else "cpu"
    nU, nV, eu, ev = synth.make_graph(spec, device=device)
    eu, ev = eu.cpu().numpy(), ev.cpu().numpy()
    m = spec["m"]
    pairs = peel_pairs_for(name, spec)
    off, adj = oracle.build_csr(nU, nV, eu, ev)
    del eu, ev
    threads = max(1, min(oracle_threads(), max(args.steps, 1)))

    def one(i):
        a, b = pairs[i % len(pairs)]
        t = time.perf_counter()
        oracle.peel(nU, nV, off, adj, a, b)
        return time.perf_counter() - t

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(one, range(args.warmup)))
        t_all = time.perf_counter()
        times = list(ex.map(one, range(args.steps)))
        wall = time.perf_counter() - t_all
    value = len(times) * m / wall / 1e9
    cpu = {"value": round(value, 4), "unit": "GTEPS", "cores": threads, "kind": "oracle",
           "sample": "%d oracle peels (one per step, rotating over %s), %d at a time in host threads, each "
                     "single-threaded; mean %.2f s per peel; CSR build excluded"
                     % (len(times), pairs, threads, statistics.mean(times) if times else 0.0)}
    cpu.update(cpu_info())
    return {
        "impl": "reference", "metric": "(alpha,beta)-core peel GTEPS", "value": round(value, 4), "unit": "GTEPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(wall / max(len(times), 1) * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": name, "graph": describe(spec, name), "queries_per_step": [list(p) for p in pairs],
                   "parallelism": "single"},
        "cpu_baseline": cpu,
        "e2e": {"value": round(value, 4), "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "timed_wall_s": round(wall, 3),
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="billion-100Mx50M-1500M")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="skip the autotuner (library defaults)")
    ap.add_argument("--no-gccplus", action="store_true", help="skip the GCC+ (core-number pruned) leg")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched grid beside the single peel")
    ap.add_argument("--serve-ops", type=int, default=0, help="updates per rate (default: the workload's)")
    ap.add_argument("--scope-ops", type=int, default=300,
                    help="serving: updates also answered with the paper's component scope (0: skip)")
    ap.add_argument("--param", action="append", default=[], help="library parameter name=value (repeatable)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    rank, world, local = dist_info()
    import torch
    dist_init(world, "nccl" if torch.cuda.is_available() else "gloo")
    if args.impl == "reference":
        line = run_reference(args, rank, world, local)
    else:
        from paper_2606_07148_gb300.buildlib import build
        if rank == 0:
            build()
        barrier(world)
        if args.workload.startswith("batch") or args.workload == "billion-batch":
            line = run_batch(args, rank, world, local)
        elif args.workload.startswith("sweep"):
            line = run_sweep(args, rank, world, local)
        elif args.workload.startswith("serve"):
            line = run_serve(args, rank, world, local)
        else:
            line = run_peel(args, rank, world, local)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
