#!/usr/bin/env python
"""Benchmark of incremental betweenness centrality on one GB300.

Default workload: undirected Barabasi-Albert graph, n = 16384, 8 edges per new vertex
(m = 131,036 edges), weights U[1,100], and a seeded stream of 1024 incremental updates
(half edge updates -- half new edges, half weight decreases --, half vertex updates on
2..16 incident edges).  int32 distances, uint64 path counts, fp64 dependencies and BC.

A "step" applies the next ``--per-step`` updates of the stream (each update is the
whole hot path: Algorithm 4 passes, the rank-1 pass of Lemma 2 / 4, DAG rebuild and
re-accumulation of every changed source, BC update).  Reported:
  value  updates/s, device time (CUDA events on the library's stream) of K steps whose
         update batch is already staged in device memory;
  e2e    the same K steps through the public C-ABI call with host buffers (one
         bc_apply_updates call per step, the updates copied to the device inside the
         call), plus a read of the BC vector after each step; p50/p99 latency per
         update and the rate of one synchronous call per update from a second pass;
  roofline of the dominant kernel class (events around each launch, second pass over
         further steps), the GPU full-recompute baseline (bc_init_static on the final
         graph) and the CPU oracle on a bounded sample of sources.
With --impl reference the CPU oracle (static Brandes recomputed after an update) is
timed instead, on the same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "edge updates/sec at n=16384 vs GPU full recompute; HBM GB/s; p50/p99 ms"
UNIT = "updates/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return PEAKS_FALLBACK["hbm_gbs"], "fallback"


def int_alu_peak():
    """Integer ALU peak in Tops/s: SMs x 128 int32 lanes per SM x the maximum SM clock
    (MEASURED_PEAKS.json's sm_max_mhz, else the nominal 2070 MHz)."""
    import torch
    mhz = 2070.0
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * 128 * mhz * 1e6 / 1e12


def workload(name: str):
    from paper_1311_2147_gb300 import synth
    if name == "ba16384":
        g, ups = synth.workload_ba16384()
        return g, ups, "i32", ("BA n=16384, 8 edges/vertex (m=131036), w~U[1,100], 1024 updates: "
                               "256 new edges, 256 decreases, 512 vertex updates k~U{2..16}")
    if name == "er256":
        g, ups = synth.workload_er256()
        return g, ups, "i64", "directed ER n=256 m=2048, w~U[1,1000], 16 updates"
    if name == "complete2048":
        g, ups = synth.workload_complete2048()
        return g, ups, "i64", "complete directed n=2048, w~U{1..n^2}, 256 weight decreases"
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.lines: list[str] = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def read_traffic(profile_name: str, units_per_launch: float):
    """DRAM bytes per launch from the committed ncu summary profiles/<profile_name>.md:
    its measured bytes per unit of work (captured on a smaller case of the same kernel)
    times the units one launch of this run processes.  None when the kernel source
    changed since the capture (its sha256 no longer matches) or there is no summary."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"{profile_name}.md")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for ln in f:
            if ":" in ln and ln.strip().startswith("- "):
                k, v = ln.strip()[2:].split(":", 1)
                vals[k.strip()] = v.strip()
    src = vals.get("source_file")
    sha = vals.get("source_sha256")
    if not src or not sha or "traffic_bytes_per_unit" not in vals:
        return None
    fp = os.path.join(ROOT, src)
    if not os.path.exists(fp) or hashlib.sha256(open(fp, "rb").read()).hexdigest() != sha:
        return None
    return float(vals["traffic_bytes_per_unit"]) * units_per_launch


def cpu_oracle_sample(g, sample_sources: int, seed: int = 7, threads: int | None = None):
    """Static Brandes (the oracle as it stands) from a seeded sample of sources of ``g``.

    Returns (seconds, threads, sources).  The time is what the sample took; a full
    recompute runs n sources of the same cost, so it takes about seconds * n / sources."""
    from oracle import oracle
    from paper_1311_2147_gb300 import synth
    n = g.n
    k = min(sample_sources, n)
    srcs = np.sort(synth.Rng(seed).below(n, k)).astype(np.int32)
    cores = threads or oracle.default_threads()
    t0 = time.perf_counter()
    oracle.brandes(g, sources=srcs, want_rows=False, want_bc=True, nthreads=cores)
    return time.perf_counter() - t0, cores, k


def run_reference(args):
    """The oracle as the reference arm: each step applies the next update of the stream
    to the host graph and recomputes static Brandes from a seeded sample of
    ``--ref-sample`` sources on all host cores.  ``ms_per_step`` is the measured time of
    those steps; one step is the fraction sample/n of a full recompute, so ``value``
    (updates/s) = K * sample/n / (timed seconds)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1311_2147_gb300 import synth
    g, ups, dist, desc = workload(args.workload)
    W, K = args.warmup, args.steps
    ups = extend_stream(args.workload, g, ups, max(0, W + K - len(ups)), seed=0x5EED)
    em = synth.EdgeMap.of(g)
    times = []
    cores = k = None
    for step in range(W + K):
        synth.apply_update(em, ups[step])
        gg = em.to_graph()
        dt, cores, k = cpu_oracle_sample(gg, args.ref_sample, seed=step)
        if step >= W:
            times.append(dt)
    frac = k / g.n
    total = sum(times)
    value = K * frac / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": K, "warmup": W, "ms_per_step": 1e3 * total / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64/u64/f64", "data": "synthetic",
            "config": {"workload": desc, "updates_per_step": frac,
                       "step": f"one update applied to the host graph, then static Brandes from {k} of "
                               f"{g.n} sources (a fraction {frac:.4g} of one full recompute)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: the next update, then static Brandes from {k} seeded sources "
                                       f"of the updated graph on {cores} threads ({1e3 * total / K:.0f} ms "
                                       f"measured per step)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


SCAN_UPDATES = 8   # updates kept back for the full rank-1 pass (roofline_scan)


def plan_steps(stream_len: int, per_step: int, warmup: int, steps: int, reserve: int = SCAN_UPDATES):
    """Updates per step U and how many updates to draw beyond the configured stream.

    The run consumes W warm-up steps, K timed steps and K profiled steps of U updates
    each, then ``reserve`` updates for the full rank-1 pass.  U is the requested
    ``per_step`` when that fits the stream, else the largest U that does; when even
    U = 1 does not fit, the stream is continued (``extra`` further updates drawn by
    the same recipe on the graph the stream leaves).  Never fails for W, K >= 1."""
    slots = warmup + 2 * steps
    if slots <= 0:
        raise ValueError("warmup + 2 * steps must be positive")
    fit = (stream_len - reserve) // slots
    U = max(1, min(per_step, fit))
    extra = max(0, slots * U + reserve - stream_len)
    return U, extra


def extend_stream(name: str, g, ups, extra: int, seed: int):
    """``ups`` continued by ``extra`` updates of the workload's own mix, drawn on the
    graph the stream leaves (BA: half edge updates, half vertex updates, w in [1,100];
    ER: half new edges, half decreases, w in [1,1000]; complete: decreases only)."""
    from paper_1311_2147_gb300 import synth
    if extra <= 0:
        return ups
    gl = synth.apply_updates(g, ups)
    if name == "ba16384":
        ne = (extra + 1) // 2
        more = synth.update_stream(gl, (ne + 1) // 2, ne // 2, extra - ne, seed, 1, 100)
    elif name == "er256":
        more = synth.update_stream(gl, (extra + 1) // 2, extra // 2, 0, seed, 1, 1000)
    else:
        more = synth.update_stream(gl, 0, extra, 0, seed, 1, gl.n * gl.n)
    return list(ups) + more


def per_class_rates(dev_ms, kinds):
    """Per-update device times split by class: edge / vertex updates, and no-ops (an
    update that changes no pair) against effective ones.  Each class: count, rate
    (updates per second of its own device time), mean and p50/p99 of the device time."""
    out = {}
    groups = {"edge": [], "vertex": [], "noop": [], "effective": [], "all": []}
    for ms, (kind, noop) in zip(dev_ms, kinds):
        groups[kind].append(ms)
        groups["noop" if noop else "effective"].append(ms)
        groups["all"].append(ms)
    for k, v in groups.items():
        if not v:
            continue
        out[k] = {"count": len(v), "updates_per_s": 1e3 * len(v) / sum(v), "mean_ms": float(np.mean(v)),
                  "p50_ms": float(np.percentile(v, 50)), "p99_ms": float(np.percentile(v, 99))}
    return out


def max_over_ranks(x: float, dist=None, device: str = "cuda") -> float:
    """The largest x over all ranks of the process group (x itself on one process)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, t_max_s: float) -> float:
    """Whole-job throughput of replicas with the same work per rank: every rank's units
    over the slowest rank's time."""
    return world * units_per_rank / t_max_s


def run_ours(args):
    import torch
    from paper_1311_2147_gb300 import binding, synth
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    binding.load()
    g, ups, dtype, desc = workload(args.workload)
    n = g.n
    W, K = args.warmup, args.steps
    stream_len = len(ups)
    U, extra_ups = plan_steps(stream_len, args.per_step, W, K)
    ups = extend_stream(args.workload, g, ups, extra_ups, seed=0x5EED + extra_ups)
    sl = [ups[i * U:(i + 1) * U] for i in range((W + 2 * K))]
    sd = 4 if dtype == "i32" else 8
    stream = torch.cuda.Stream()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    # ---------------- value: device time, update batches resident before timing
    A = binding.BCGraph(g, dist=dtype, stream=stream.cuda_stream)
    for i in range(W):
        rc, done = A.bc_apply_updates(sl[i])
        assert rc == 0, A.last_error()
    timed = [u for s in sl[W:W + K] for u in s]
    assert A.bc_stage_updates(timed) == 0
    info0 = A.bc_get_info()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(local) as clk:
        e0.record(stream)
        rc, done = A.bc_run_staged()
        e1.record(stream)
        assert rc == 0 and done == len(timed), A.last_error()
        assert A.bc_synchronize() == 0, A.last_error()
        barrier()
    dev_ms = e0.elapsed_time(e1)
    info1 = A.bc_get_info()
    launches = info1["kernel_launches"] - info0["kernel_launches"]
    t_max = max_over_ranks(dev_ms, dist)
    value = job_rate(len(timed), world, t_max / 1e3)

    # ---------------- per-kernel-class profile over the next K steps (events per launch)
    A.bc_set_option("profile", 1)
    A.bc_get_profile(reset=True)
    infop0 = A.bc_get_info()
    prof_updates = [u for s in sl[W + K:W + 2 * K] for u in s]
    rc, done = A.bc_apply_updates(prof_updates)
    assert rc == 0, A.last_error()
    prof = A.bc_get_profile(reset=True)
    infop1 = A.bc_get_info()
    A.bc_set_option("profile", 0)
    dinfo = {k: infop1[k] - infop0[k] for k in infop1 if isinstance(infop1[k], int)}
    d_rows_acc, d_rows_scan = dinfo["rows_reaccumulated"], dinfo["rows_scanned"]
    d_low, d_tie = dinfo["pairs_lowered"], dinfo["pairs_tied"]
    d_full, d_pair_rows, d_pair_tgts = dinfo["rows_full"], dinfo["pair_rows"], dinfo["pair_targets"]
    d_walk_pairs, d_walk_vtx, d_walk_arcs = dinfo["walk_pairs"], dinfo["walk_vertices"], dinfo["walk_arcs"]
    # algorithmic HBM bytes per kernel class over the profiled steps
    alg_bytes = {
        # rank-1 pass: read d of every scanned pair, sigma read+write on ties, d+sigma
        # written where the distance drops
        "scan": d_rows_scan * n * sd + d_tie * 16 + d_low * (sd + 8),
        # accumulation (the rows over the target cap): d row, sigma row, new delta row
        "accumulate": d_full * n * (sd + 8 + 8),
        # BC: the re-accumulated delta rows are read twice (before and after); with pair
        # corrections only the full rows are, and per update the fixed-point column
        # changes are read and BC (hi, lo) read and written (16 bytes each per column)
        "bc_rows": (2 * d_full * n * 8 + len(prof_updates) * n * 48) if d_pair_rows
        else 2 * d_rows_acc * n * 8,
    }
    # pair corrections: per (row, changed target, column) one add and one compare for
    # each of the two states (integer ALU work; the rows come from L2)
    alu_ops = {"pair_corrections": 4 * d_pair_tgts * n}
    peak, peak_kind = load_peaks()
    int_peak = int_alu_peak()
    if d_walk_pairs:
        # pair corrections by DAG walks: per E* arc examined the arc (8 B) and d(s,x) (sd B);
        # per vertex found its segment bounds (8 B), two path counts (16 B), its list entry
        # written and read back (8 B) and its buffer entry written and read (8 B)
        alg_bytes["pair_corrections"] = d_walk_arcs * (8 + sd) + d_walk_vtx * (8 + 16 + 8 + 8)
        alu_ops.pop("pair_corrections")
    dom = max(prof, key=lambda c: prof[c][0])
    dom_ms, dom_launches = prof[dom]
    roof = None
    if dom == "pair_corrections" and d_walk_pairs and dom_ms > 0 and dom_launches > 0:
        kl = len(prof_updates)
        achieved = alg_bytes[dom] / (dom_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel_class": dom,
                "kernel": "k_walk_units + k_walk_rows_hash + k_walk_rows (DAG walks; with k_pair_plan, k_pair_weights)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                "alg_bytes_per_launch": alg_bytes[dom] / kl,
                "traffic": read_traffic("walks_ba8192", (d_walk_arcs + d_walk_vtx) / kl),
                "launches": kl, "avg_launch_ms": dom_ms / kl,
                "note": "latency-bound gathers along shortest-path DAGs; bytes counted per arc and vertex visited"}
    elif dom in alu_ops and dom_ms > 0 and dom_launches > 0:
        kl = dom_launches // 3 or 1   # k_pair_plan, k_pair_weights, k_pairdep per update
        achieved = alu_ops[dom] / (dom_ms / 1e3) / 1e12
        roof = {"bound": "alu", "kernel_class": dom, "kernel": "k_pairdep (with k_pair_plan, k_pair_weights)",
                "achieved": achieved, "peak": int_peak, "unit": "Tops/s (int32)", "frac": achieved / int_peak,
                "peak_kind": "derived: SMs x 128 int32 lanes x max SM clock",
                "alg_ops_per_launch": alu_ops[dom] / kl,
                "traffic": read_traffic("pair_corrections_ba8192", d_pair_rows * n / kl),
                "launches": kl, "avg_launch_ms": dom_ms / kl}
    elif dom in alg_bytes and dom_launches > 0 and dom_ms > 0:
        per_launch = alg_bytes[dom] / dom_launches
        achieved = alg_bytes[dom] / (dom_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel_class": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": peak_kind,
                "alg_bytes_per_launch": per_launch, "traffic": None,
                "launches": dom_launches, "avg_launch_ms": dom_ms / dom_launches}
    classes = {c: {"ms": prof[c][0], "launches": prof[c][1],
                   "gbs": (alg_bytes[c] / (prof[c][0] / 1e3) / 1e9) if c in alg_bytes and prof[c][0] > 0 else None}
               for c in prof}

    # ---------------- the n x n update kernel over every row (the paper's all-pairs
    # Step 2), on the same state: HBM roofline of the rank-1 pass
    roof_scan = None
    extra = ups[(W + 2 * K) * U:(W + 2 * K) * U + SCAN_UPDATES]
    if extra:
        A.bc_set_option("full_scan", 1)
        A.bc_set_option("profile", 1)
        A.bc_get_profile(reset=True)
        tot_ms = tot_b = 0.0
        tot_nl = tot_rows = 0
        per_upd = []
        for up in extra:   # one update at a time: per-update figures beside the totals
            i0 = A.bc_get_info()
            rc, _ = A.bc_apply_updates([up])
            assert rc == 0, A.last_error()
            pf = A.bc_get_profile(reset=True)
            i1 = A.bc_get_info()
            ms, nl = pf["scan"]
            rows = i1["rows_scanned"] - i0["rows_scanned"]
            low, tie = i1["pairs_lowered"] - i0["pairs_lowered"], i1["pairs_tied"] - i0["pairs_tied"]
            b = rows * n * sd + tie * 16 + low * (sd + 8)
            if nl:
                per_upd.append({"kind": up[0], "launches": nl, "avg_launch_ms": ms / nl,
                                "gbs": b / (ms / 1e3) / 1e9, "pairs_changed": low + tie})
            tot_ms += ms
            tot_b += b
            tot_nl += nl
            tot_rows += rows
        A.bc_set_option("profile", 0)
        A.bc_set_option("full_scan", 0)
        if tot_ms > 0 and tot_nl > 0:
            achieved = tot_b / (tot_ms / 1e3) / 1e9
            roof_scan = {"bound": "hbm", "kernel": "k_scan_cs, every row (full pass)", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                         "alg_bytes_per_launch": tot_b / tot_nl,
                         "traffic": read_traffic("scan_ba8192_fullscan", tot_rows * n / tot_nl),
                         "launches": tot_nl, "avg_launch_ms": tot_ms / tot_nl, "updates": len(extra),
                         "median_update_gbs": float(np.median([u["gbs"] for u in per_upd])),
                         "per_update": per_upd}
    A.close()

    # ---------------- e2e through the C-ABI with host buffers
    # Timed pass: every step is one bc_apply_updates call with the step's updates in host
    # memory (copied to the device inside the call) and a read of the BC vector after it,
    # on a fresh handle brought to the same state by the warm-up steps.  Latency pass: the
    # same steps on another fresh handle, one call per update, timed around each call
    # (p50/p99 per update, and the rate of that synchronous use), with the device time of
    # every update from events around its call for the per-class rates.
    e2e = None
    per_class = None
    lat = []
    if not args.no_e2e:
        B = binding.BCGraph(g, dist=dtype, stream=stream.cuda_stream)
        for i in range(W):
            rc, _ = B.bc_apply_updates(sl[i])
            assert rc == 0
        enc = [binding.encode_updates(s) for s in sl[W:W + K]]
        h2d = sum(rec.nbytes + ed.nbytes for rec, ed in enc)
        d2h = 0
        barrier()
        t0 = time.perf_counter()
        for rec, ed in enc:
            rc, _ = B.bc_apply_updates((rec, ed))
            assert rc == 0, B.last_error()
            scores = B.bc_get_scores()
            d2h += 2 * scores.nbytes
        barrier()
        wall = max_over_ranks(time.perf_counter() - t0, dist)
        B.close()
        C = binding.BCGraph(g, dist=dtype, stream=stream.cuda_stream)
        for i in range(W):
            rc, _ = C.bc_apply_updates(sl[i])
            assert rc == 0
        evs = []
        kinds = []
        call_s = 0.0
        for s in sl[W:W + K]:
            for up in s:
                rec, ed = binding.encode_updates([up])
                ea = torch.cuda.Event(enable_timing=True)
                eb = torch.cuda.Event(enable_timing=True)
                noop0 = C.bc_get_info()["noop_updates"]
                ta = time.perf_counter()
                ea.record(stream)
                rc, _ = C.bc_apply_updates((rec, ed))
                eb.record(stream)
                dt = time.perf_counter() - ta
                lat.append(1e3 * dt)
                call_s += dt
                assert rc == 0, C.last_error()
                evs.append((ea, eb))
                kinds.append((up[0], C.bc_get_info()["noop_updates"] > noop0))
            ta = time.perf_counter()
            C.bc_get_scores()
            call_s += time.perf_counter() - ta
        dev = [ea.elapsed_time(eb) for ea, eb in evs]
        e2e = {"value": job_rate(len(timed), world, wall), "unit": UNIT, "h2d_bytes_per_step": h2d // K,
               "d2h_bytes_per_step": d2h // K, "p50_ms": float(np.percentile(lat, 50)),
               "p99_ms": float(np.percentile(lat, 99)),
               "calls": "one bc_apply_updates per step; p50/p99 from one call per update",
               "per_update_calls_value": len(timed) / call_s}
        per_class = per_class_rates(dev, kinds)
        C.close()

    # ---------------- complete graph: the "effective decreases" variant (w' <= d(u,v),
    # d read from the handle's own state through the C-ABI), per-update device times
    effective = None
    if args.workload == "complete2048" and not args.no_e2e:
        C = binding.BCGraph(g, dist=dtype, stream=stream.cuda_stream)
        rows = {}

        def dist_uv(a_, b_):
            if a_ not in rows:
                rows[a_] = C.bc_get_rows(int(a_), 1, want=("d",))[0][0]
            return int(rows[a_][b_])
        dec = synth.effective_decreases(g, dist_uv, args.effective_updates, 0xEFFE)
        devs, kinds = [], []
        for up in dec:
            ea = torch.cuda.Event(enable_timing=True)
            eb = torch.cuda.Event(enable_timing=True)
            noop0 = C.bc_get_info()["noop_updates"]
            ea.record(stream)
            rc, _ = C.bc_apply_updates([up])
            eb.record(stream)
            assert rc == 0, C.last_error()
            kinds.append((up[0], C.bc_get_info()["noop_updates"] > noop0))
            devs.append((ea, eb))
        torch.cuda.synchronize()
        effective = {"updates": len(dec), "draw": "w' ~ U[1, min(w-1, d(u,v))] on random existing arcs",
                     "per_class": per_class_rates([a_.elapsed_time(b_) for a_, b_ in devs], kinds)}
        C.close()

    # ---------------- baselines: GPU full recompute and the CPU oracle (rank 0 only)
    gpu_full = None
    cpu = None
    if rank == 0 and not args.no_baselines:
        gfin = synth.apply_updates(g, ups[:(W + 2 * K) * U])
        ms = []
        for _ in range(args.recompute_runs):
            C = binding.BCGraph(gfin, dist=dtype, stream=stream.cuda_stream)
            ms.append(C.bc_get_info()["last_init_ms"])
            C.close()
        med = statistics.median(ms)
        ms_all = []
        for _ in range(args.recompute_runs):
            C = binding.BCGraph(gfin, dist=dtype, stream=stream.cuda_stream, static_all_arcs=True)
            ms_all.append(C.bc_get_info()["last_init_ms"])
            C.close()
        gpu_full = {"ms": med, "runs": ms, "updates_per_s": 1e3 / med,
                    "incremental_speedup": value / world / (1e3 / med),
                    "static": "searches restricted to E* as it becomes known (Algorithm 6 step 1)",
                    "all_arcs_ms": statistics.median(ms_all),
                    "all_arcs_note": "the same static computation searching every arc (BC_STATIC_ALL_ARCS)"}
        if world == 1:
            dt, cores, k = cpu_oracle_sample(gfin, args.cpu_sample)
            dt1, _, k1 = cpu_oracle_sample(gfin, args.cpu_sample_one_core, seed=8, threads=1)
            cpu = {"value": k / n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"static Brandes from {k} seeded sources of the final graph, measured "
                             f"{dt:.2f} s on {cores} threads; value = (k/n) / time, one full "
                             f"recompute per update",
                   "one_core": {"value": k1 / n / dt1, "unit": UNIT, "cores": 1,
                                "sample": f"{k1} seeded sources on one thread, measured {dt1:.2f} s"}}

    if rank == 0:
        rows_per_upd = (info1["rows_reaccumulated"] - info0["rows_reaccumulated"]) / len(timed)
        per_update = {k: (info1[k] - info0[k]) / len(timed)
                      for k in ("rows_reaccumulated", "rows_full", "pair_rows", "pair_targets", "walk_pairs",
                                "walk_vertices", "walk_arcs", "rows_scanned",
                                "pairs_lowered", "pairs_tied", "estar_moves", "estar_rebuilds")}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": t_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int32/u64/f64" if dtype == "i32" else "int64/u64/f64", "data": "synthetic",
                "config": {"workload": desc, "updates_per_step": U,
                           "stream": {"configured_updates": stream_len, "drawn_beyond": extra_ups,
                                      "warmup_updates": W * U, "timed_updates": K * U,
                                      "profiled_updates": K * U, "full_pass_updates": SCAN_UPDATES},
                           "l2": f"state {n * n * (sd + 16 + (0 if g.directed else sd + 8)) / 1e9:.2f} GB per graph > 129 MB L2; no flush",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "e2e": e2e, "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu,
                "clocks": clk.summary(), "gpu_full_recompute": gpu_full,
                "latency_ms": {"p50": e2e["p50_ms"], "p99": e2e["p99_ms"]} if e2e else None,
                "roofline_scan": roof_scan,
                "classes": classes, "rows_per_update": rows_per_upd, "per_update": per_update,
                "per_class": per_class, "effective_decreases": effective}
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """Batched workload: 512 graphs, n log-uniform in [64, 2048] (even index directed ER
    with out-degree 8, odd undirected BA(8)), w ~ U[1,1000]; a step applies 8 edge
    updates to every graph (half new edges, half decreases) in one CUDA graph launch."""
    import torch
    from paper_1311_2147_gb300 import autotune, binding, synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    binding.load()
    W, K, per = args.warmup, args.steps, 8
    tune_steps = autotune.steps_needed()
    total_steps = tune_steps + W + K
    t0 = time.perf_counter()
    fam = synth.workload_batch(count=args.batch_graphs, n_updates=per, rounds=total_steps)
    gen_s = time.perf_counter() - t0
    graphs = [binding.BCGraph(g, dist="i32") for g, _ in fam]
    # baseline: one static recompute (bc_init_static) of every graph per update it takes
    init_ms = [h.bc_get_info()["last_init_ms"] for h in graphs]
    stream = torch.cuda.Stream()
    batch = binding.BCBatch(graphs, stream=stream.cuda_stream)
    step_i = [0]

    def next_step():
        k = step_i[0]
        step_i[0] += 1
        lists = [ups[k * per:(k + 1) * per] for _, ups in fam]
        if any(len(u) != per for u in lists):
            raise RuntimeError(f"batch step {k} is past the generated stream ({total_steps} steps)")
        return lists

    n_max = max(g.n for g, _ in fam)
    key = autotune.cache_key(len(fam), n_max, "i32")
    tiles, trials = autotune.tune(batch, next_step, key=key, use_cache=False)
    for _ in range(W):
        rc, _ = batch.bc_batch_apply(next_step())
        assert rc == 0, batch.last_error()
    ms = []
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for _ in range(K):
            rc, _ = batch.bc_batch_apply(next_step())
            assert rc == 0, batch.last_error()
            ms.append(batch.bc_batch_last_ms())
    total_ms = sum(ms)
    updates = K * per * len(fam)
    sum_n2 = sum(g.n * g.n for g, _ in fam)
    line = {"metric": "updates/sec over a batch of graphs (one CUDA graph launch per step)",
            "value": updates / (total_ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": W,
            "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32/u64/f64", "data": "synthetic",
            "config": {"workload": f"{len(fam)} graphs, n log-uniform in [64,2048] (max {n_max}), "
                                   f"half directed ER out-degree 8, half undirected BA(8), w~U[1,1000], "
                                   f"8 edge updates per graph per step",
                       "sum_n2": sum_n2, "state_gb": sum_n2 * 20 / 1e9, "tiles": tiles,
                       "autotune_trials": trials, "generation_s": gen_s},
            "gpu_full_recompute": {"sum_init_ms": sum(init_ms), "updates_per_s": len(fam) / (sum(init_ms) / 1e3),
                                   "note": "bc_init_static of every graph once per update of that graph "
                                           "(the sum of the per-graph static times at creation)",
                                   "incremental_speedup": (updates / (total_ms / 1e3)) /
                                                          (len(fam) / (sum(init_ms) / 1e3))},
            "clocks": clk.summary()}
    print(json.dumps(line))
    return 0


def run_serve(args):
    """Serving workload: 64 resident graphs, n log-uniform in [1024, 8192], alternately
    directed ER (out-degree 8) and undirected BA(8), w ~ U[1,100]; requests are edge
    updates or vertex updates on 2..16 edges (half each) for uniformly drawn graphs.
    Saturated throughput is measured closed-loop (all requests submitted at once), then
    an open-loop Poisson stream at --serve-load x that rate gives p50/p99 latency."""
    import torch
    from paper_1311_2147_gb300 import binding, synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    binding.load()
    seed = synth.BASE_SEED + 4
    rng = synth.Rng(seed)
    G = args.serve_graphs
    ns = synth.log_uniform_n(rng, 1024, 8192, G)
    graphs = []
    for i, n in enumerate(ns):
        g = (synth.erdos_renyi_degree(n, 8, 1, 100, synth.sub_seed(seed, i)) if i % 2 == 0
             else synth.barabasi_albert(n, 8, 1, 100, synth.sub_seed(seed, i)))
        graphs.append(g)
    R = args.serve_requests
    loads = [float(x) for x in str(args.serve_loads).split(",")] if args.serve_loads else [args.serve_load]
    # requests over uniformly drawn graphs, each stream valid against its own graph:
    # R closed-loop requests, then R open-loop requests per load
    pick = rng.below(G, (1 + len(loads)) * R + 64).tolist()
    per_graph = [0] * G
    for gi in pick:
        per_graph[gi] += 1
    streams = []
    for i, g in enumerate(graphs):
        k = per_graph[i]
        ne = k // 2
        streams.append(synth.update_stream(g, ne // 2, ne - ne // 2, k - ne, synth.sub_seed(seed, 1000 + i),
                                           1, 100) if k else [])
    nxt = [0] * G
    seq = []
    for gi in pick:
        seq.append((gi, streams[gi][nxt[gi]]))
        nxt[gi] += 1
    state = sum(n * n * 20 for n in ns)
    srv = binding.BCServer(budget_bytes=int(state * 1.5) + (8 << 30), max_batch=64)
    gids = [srv.add_graph(g) for g in graphs]
    # closed loop: saturated throughput on the first R requests
    closed = seq[:R]
    t0 = time.perf_counter()
    for gi, up in closed:
        srv.submit(gids[gi], up)
    res_c = srv.drain()
    t_closed = time.perf_counter() - t0
    sat = len(closed) / t_closed
    # open loop: Poisson arrivals at each load x saturated throughput, R requests each
    runs = []
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for li, load in enumerate(loads):
            lam = load * sat
            gaps = -np.log(1.0 - synth.Rng(seed + 1 + li).unit(R)) / lam
            arrivals = np.cumsum(gaps)
            opened = seq[(1 + li) * R:(2 + li) * R]
            res = []
            t0 = time.perf_counter()
            i = 0
            while i < len(opened):
                now = time.perf_counter() - t0
                while i < len(opened) and arrivals[i] <= now:
                    gi, up = opened[i]
                    srv.submit(gids[gi], up)
                    i += 1
                r = srv.poll()
                if r.size:
                    res.append(r)
            res.append(srv.drain())
            t_open = time.perf_counter() - t0
            res = np.concatenate(res)
            lat = res["latency_ns"] / 1e6
            runs.append({"load": load, "lambda_per_s": lam, "updates_per_s": len(opened) / t_open,
                         "seconds": t_open, "requests": len(opened),
                         "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                        "max": float(lat.max())},
                         "failures": int((res["status"] != 0).sum())})
    head = min(runs, key=lambda r: abs(r["load"] - 0.8))
    st = srv.stats()
    # counters summed over the resident graphs (what explains the latency tail: updates
    # that re-accumulate many rows, E* segment moves and re-layouts)
    counters = {}
    for gid in gids:
        info = srv.graph(gid).bc_get_info()
        for k in ("updates_applied", "noop_updates", "rows_full", "estar_moves", "estar_rebuilds", "max_rows"):
            counters[k] = max(counters.get(k, 0), info[k]) if k == "max_rows" else counters.get(k, 0) + info[k]
    line = {"metric": "serving: updates/sec and p50/p99 latency over resident graphs",
            "value": head["updates_per_s"], "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": head["seconds"] * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32/u64/f64", "data": "synthetic",
            "config": {"workload": f"{G} graphs n log-uniform [1024,8192], ER/BA, w~U[1,100], "
                                   f"{R} closed-loop then {R} Poisson requests per load (half edge, half vertex k 2..16)",
                       "state_gb": state / 1e9, "saturated_updates_per_s": sat, "load": head["load"],
                       "lambda_per_s": head["lambda_per_s"]},
            "latency_ms": head["latency_ms"], "loads": runs,
            "closed_loop_failures": int((res_c["status"] != 0).sum()),
            "open_loop_failures": sum(r["failures"] for r in runs),
            "server": st, "graph_counters": counters, "clocks": clk.summary()}
    print(json.dumps(line))
    return 0


def run_ncu_case(args):
    """A small case of one kernel class for ncu captures (a few GB on the device at most):
    BA n=8192 (state 2.1 GB, above L2), static init, then either two vertex updates with
    every changed row re-accumulated (accumulation and BC rows), the first four updates
    of the stream with pair corrections by the column test (pair) or by DAG walks
    (walk), or two edge updates with the rank-1 pass over every row (the paper's
    all-pairs Step 2)."""
    from paper_1311_2147_gb300 import binding, synth
    binding.load()
    g, ups = synth.workload_ba16384(n=args.ncu_n, n_updates=64)
    bg = binding.BCGraph(g, dist="i32")
    if args.ncu_case == "scan":
        bg.bc_set_option("full_scan", 1)
        sel = [u for u in ups if u[0] == "edge"][:2]
    elif args.ncu_case == "pair":
        bg.bc_set_option("pair_walk", 0)
        sel = ups[:4]
    elif args.ncu_case == "walk":
        bg.bc_set_option("pair_walk", 1)
        sel = ups[:4]
    else:
        bg.bc_set_option("pair_updates", 0)
        sel = [u for u in ups if u[0] == "vertex"][:2]
    per_update = []
    for u in sel:
        before = bg.bc_get_info()
        rc, _ = bg.bc_apply_updates([u])
        assert rc == 0, bg.last_error()
        after = bg.bc_get_info()
        per_update.append({k: after[k] - before[k] for k in ("rows_reaccumulated", "rows_full", "pair_rows",
                                                             "pair_targets", "walk_pairs", "walk_vertices",
                                                             "walk_arcs", "rows_scanned", "pairs_lowered",
                                                             "pairs_tied")})
    print(json.dumps({"ncu_case": args.ncu_case, "n": g.n, "per_update": per_update, "info": bg.bc_get_info()}))
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--per-step", type=int, default=32)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="ba16384",
                    choices=["ba16384", "er256", "complete2048", "batch512", "serve"])
    ap.add_argument("--serve-graphs", type=int, default=64)
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-load", type=float, default=0.8)
    ap.add_argument("--serve-loads", default="0.5,0.8,0.95",
                    help="comma-separated loads (x saturated throughput) of the open-loop runs")
    ap.add_argument("--batch-graphs", type=int, default=512)
    ap.add_argument("--cpu-sample", type=int, default=4096,
                    help="sources of the all-core CPU oracle sample (cpu_baseline)")
    ap.add_argument("--cpu-sample-one-core", type=int, default=256,
                    help="sources of the one-core CPU oracle sample")
    ap.add_argument("--ref-sample", type=int, default=1024,
                    help="sources recomputed per step of the reference arm")
    ap.add_argument("--recompute-runs", type=int, default=3)
    ap.add_argument("--effective-updates", type=int, default=64,
                    help="complete-graph workload: effective decreases in the variant run")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-baselines", action="store_true")
    ap.add_argument("--ncu-case", choices=["accumulate", "pair", "walk", "scan"], default=None,
                    help="run only a small case of one kernel class (for ncu captures)")
    ap.add_argument("--ncu-n", type=int, default=8192)
    args = ap.parse_args()
    if args.ncu_case:
        return run_ncu_case(args)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch512":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
