"""Benchmark: SpMV GB/s of the selected variant vs plain CSR on the four-class
synthetic set, on one GB300 (or N replicas under torchrun).

A step is one SpMV y = A x with the selected variant on each of the four
matrices (27-point stencil 128^3, random columns 4M x 16, Zipf(1.8) rows 1M
with a 200k row, 8M rows x 2).  Selection (features, profiling runs, rule)
and preparation happen once before the timed region, as in an iterative
solver; their cost is reported in SpMVs of plain CSR.  Every matrix is larger
than the 129 MB L2, so consecutive SpMVs do not reuse A from L2.

`--impl reference` times the CPU oracle (sequential FP64 CSR SpMV, one host
core) on a bounded row sample of the same matrices.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = ("four-class synthetic set, FP64 values ~U[-1,1], int32 indices: 27-pt 3D stencil "
            "128^3 (2.1M rows, 55.7M nnz); random uniform columns 4M rows x 16; Zipf(1.8) row "
            "lengths 1M rows, max 200k; 8M rows x 2 nnz/row")
METRIC = "SpMV GB/s (% of HBM peak) selected vs plain CSR; speedup; selector cost in SpMVs"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _traffic(variant: str, matrix: str):
    """DRAM bytes per launch recorded from ncu for this kernel, or None when
    no capture exists or its sources changed since."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(f"{variant}@{matrix}")
        if not rec:
            return None
        for path, prefix in rec["sources"].items():
            with open(os.path.join(ROOT, path), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest()[:len(prefix)] != prefix:
                    return None
        return int(rec["dram_bytes"])
    except Exception:
        return None


def _models(sp):
    """The committed selector networks: the first level (variant) and the
    second level (SLICED's launch configuration), when present."""
    data = os.path.join(ROOT, "paper_1511_02494_gb300", "data")
    first, second = os.path.join(data, "selector_mlp.bin"), os.path.join(data, "selector_sliced_mlp.bin")
    model = sp.spmv_model_load(first) if os.path.exists(first) else None
    sub = sp.spmv_model_load(second) if model is not None and os.path.exists(second) else None
    return model, sub


def _host() -> str:
    """CPU of the host the oracle runs on: architecture, model, core count."""
    import platform
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return f"{platform.machine()} {model} x{os.cpu_count()}".replace("  ", " ")


def _max_over_ranks(v: float, ws: int, device) -> float:
    """The slowest rank's value (the job's time); identity on one rank."""
    if ws <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_gbs(bytes_per_step_per_rank: int, steps: int, ws: int, total_ms: float) -> float:
    """Whole-job throughput: the bytes every replica processed over the
    slowest replica's time (weak scaling: each rank runs the full workload)."""
    return bytes_per_step_per_rank * steps * ws / (total_ms * 1e-3) / 1e9


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.proc, self.lines = index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU side
SAMPLE_BLOCK = 256  # rows per block of the CPU row sample


def _row_sample(A, stride: int, block: int = SAMPLE_BLOCK):
    """Every stride-th block of `block` consecutive rows, over the whole
    matrix (a bounded CPU sample that sees every part of it: the stencil's
    boundary rows, the Zipf matrix's long and short rows alike)."""
    import numpy as np
    import torch
    import synth
    rp = A.rowptr.to(torch.int64).numpy()
    starts = np.arange(0, A.n_rows, block * stride)
    ends = np.minimum(starts + block, A.n_rows)
    rows = np.concatenate([np.arange(s, e) for s, e in zip(starts, ends)])
    lens = rp[rows + 1] - rp[rows]
    idx = np.concatenate([np.arange(rp[s], rp[e]) for s, e in zip(starts, ends)])
    rowptr = torch.from_numpy(np.concatenate([[0], np.cumsum(lens)]).astype(np.int32))
    idx_t = torch.from_numpy(idx)
    return synth.HostCSR(len(rows), A.n_cols, rowptr, A.colind[idx_t].clone(), A.val[idx_t].clone(),
                         A.name)


def _slice_bytes(S):
    return 12 * S.nnz + 4 * (S.n_rows + 1) + 16 * S.n_rows


def _sample_desc(stride: int) -> str:
    return (f"every {stride}th block of {SAMPLE_BLOCK} rows over the whole of each of the 4 matrices "
            f"(1/{stride} of the rows)")


def cpu_oracle_rate(mats, budget_s: float, stride: int = 16, trials: int = 5):
    """GB/s of the oracle's sequential SpMV on strided row samples (one host
    core): the median of `trials` trials, each as many passes over the four
    samples as fit in budget_s / trials."""
    import statistics
    import oracle
    import synth
    slices = [_row_sample(A, stride) for A in mats]
    xs = [synth.uniform_vector(A.n_cols, 0).numpy() for A in mats]
    oracle.spmv(slices[0], xs[0])  # load / warm
    rates, passes = [], 0
    for _ in range(trials):
        tb, tt = 0, 0.0
        t_end = time.perf_counter() + budget_s / trials
        while True:
            for S, x in zip(slices, xs):
                t0 = time.perf_counter()
                oracle.spmv(S, x)
                tt += time.perf_counter() - t0
                tb += _slice_bytes(S)
            passes += 1
            if time.perf_counter() > t_end:
                break
        rates.append(tb / tt / 1e9)
    sample = (f"oracle sequential FP64 CSR SpMV over {_sample_desc(stride)}; median of {trials} "
              f"trials, {passes} passes in all")
    return statistics.median(rates), sample, rates


def cpu_table2_rate(mats, reps: int = 5):
    """The paper's own CPU method on the host cores (baseline only): the
    OpenMP restatement of its multithreaded CSR baseline and of Table 2's
    four optimizations, every form timed on the full matrices (median of
    `reps` runs after one warm-up).  value: the step with each matrix in its
    fastest Table 2 form; base_value: the unoptimized baseline."""
    import statistics
    import baseline
    import synth
    per, t_best, t_base, nbytes = {}, 0.0, 0.0, 0
    for A in mats:
        M = baseline.Matrix(A)
        M.prepare_delta()
        x = synth.uniform_vector(A.n_cols, 0).numpy()
        y = None
        ms = {}
        for form in baseline.FORMS:
            y = baseline.spmv(form, M, x, y)
            ts = []
            for _ in range(reps):
                t0 = time.perf_counter()
                baseline.spmv(form, M, x, y)
                ts.append(time.perf_counter() - t0)
            ms[form] = statistics.median(ts) * 1e3
        best = min((f for f in baseline.FORMS if f != "base"), key=lambda f: ms[f])
        per[A.name] = {"ms": {f: round(v, 3) for f, v in ms.items()}, "fastest_table2": best}
        t_best += ms[best]
        t_base += ms["base"]
        nbytes += A.min_bytes()
    return {"value": round(nbytes / (t_best * 1e-3) / 1e9, 2), "unit": "GB/s",
            "cores": baseline.threads(),
            "kind": "baseline only: OpenMP restatement of Table 2's optimizations (Section 3.3), "
                    "the fastest per matrix",
            "base_value": round(nbytes / (t_base * 1e-3) / 1e9, 2),
            "sample": f"the full four matrices, median of {reps} runs per form and matrix",
            "host": _host(), "per_matrix": per}


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return 0
    import synth
    mats = synth.four_class_set()
    import oracle
    import statistics
    stride = 16
    slices = [_row_sample(A, stride) for A in mats]
    xs = [synth.uniform_vector(A.n_cols, 0).numpy() for A in mats]
    for _ in range(args.warmup):
        for S, x in zip(slices, xs):
            oracle.spmv(S, x)
    step_s = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for S, x in zip(slices, xs):
            oracle.spmv(S, x)
        step_s.append(time.perf_counter() - t0)
    dt = sum(step_s)
    step_bytes = sum(_slice_bytes(S) for S in slices)
    gbs = step_bytes * args.steps / dt / 1e9
    median_gbs = step_bytes / statistics.median(step_s) / 1e9
    sample = f"{_sample_desc(stride)}, per step"
    line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample, "cores": 1},
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": sample, "host": _host(),
                             "median_step_value": median_gbs},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU side
def run_ours(args):
    import numpy as np
    import torch
    import paper_1511_02494_gb300 as sp
    import synth

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1511_02494_gb300.build import build
    if rank == 0:
        build()
    if ws > 1:
        torch.distributed.barrier()
    sp.lib()
    peak, peak_kind = _peaks()
    stream = torch.cuda.current_stream()

    mats = synth.four_class_set(scale=args.scale)
    dev = [sp.DeviceCSR.from_host(A) for A in mats]
    xs = [synth.uniform_vector(A.n_cols, 0).cuda() for A in mats]
    ys = [torch.empty(A.n_rows, dtype=torch.float64, device="cuda") for A in mats]

    def time_spmv(P, x, y, reps=20, warm=3, fn=None):
        fn = fn or (lambda: sp.spmv(P, x, y))
        for _ in range(warm):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    model, sub = _models(sp)
    per = []
    candidates = [("scalar", {}), ("subwarp", {}), ("stream", {}), ("merge", {}),
                  ("dynamic", {}), ("latency", {}), ("compressed", {}), ("sliced", {})]
    for A, dA, x, y in zip(mats, dev, xs, ys):
        rec = {"matrix": A.name, "n_rows": A.n_rows, "nnz": A.nnz}
        # plain CSR
        P0 = sp.spmv_prepare(dA, sp.make_choice("scalar"))
        t_plain = time_spmv(P0, x, y)
        rec["plain_ms"] = t_plain
        rec["min_bytes"] = P0.info().min_bytes
        # feature extraction + learned selector (the paper's lightweight path)
        sp.spmv_features(dA)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f = sp.spmv_features(dA)
        ch_model = sp.spmv_select_model_refined(f, model, sub) if model is not None else None
        rec["features_ms"] = (time.perf_counter() - t0) * 1e3
        # profiling runs + rule (Section 3.2.1)
        t0 = time.perf_counter()
        prof = sp.spmv_profile(dA, x, reps=3)
        ch_rule = sp.spmv_select(features=f, profile=prof)
        rec["profile_select_ms"] = (time.perf_counter() - t0) * 1e3
        rec["profile"] = {k: round(v, 4) if isinstance(v, float) else v
                          for k, v in prof.as_dict().items()}
        rec["class"] = sp.CLASSES[ch_rule.cls]
        rec["variant_rule"] = sp.VARIANTS[ch_rule.variant]
        ch = ch_model if ch_model is not None else ch_rule
        rec["variant"] = sp.VARIANTS[ch.variant]
        t0 = time.perf_counter()
        P = sp.spmv_prepare(dA, ch)
        rec["prepare_ms"] = (time.perf_counter() - t0) * 1e3
        rec["choice"] = ch
        rec["selected_min_bytes"] = P.info().min_bytes
        # the profiling rule's own choice (its class's variant and launch
        # configuration), timed alone like the variants below
        Pr = sp.spmv_prepare(dA, ch_rule)
        ir = Pr.info()
        rec["rule_launch"] = {"threads_per_row": ir.threads_per_row, "block_nnz": ir.block_nnz,
                              "items_per_warp": ir.items_per_warp}
        rec["rule_ms"] = time_spmv(Pr, x, y, reps=10)
        Pr.free()
        rec["selected_alone_ms"] = time_spmv(P, x, y, reps=10)
        inf = P.info()
        rec["launch"] = {"threads_per_row": inf.threads_per_row, "block_nnz": inf.block_nnz,
                         "items_per_warp": inf.items_per_warp, "index_bytes": inf.index_bytes,
                         "uniform_len": inf.uniform_len}
        # every variant, for the "best possible" comparison
        times = {}
        for v, kw in ([] if args.no_variant_sweep else candidates):
            Pv = P if v == rec["variant"] else sp.spmv_prepare(dA, sp.make_choice(v, **kw))
            times[v] = time_spmv(Pv, x, y, reps=10)
            if Pv is not P:
                Pv.free()
        rec["variant_ms"] = {k: round(v, 5) for k, v in times.items()}
        rec["best_variant"] = min(times, key=times.get) if times else None
        # the cost of this matrix's x gathers alone in CSR order (spmv_gather_probe)
        gsum = torch.empty(1, dtype=torch.int64, device="cuda")
        rec["gather_ms"] = time_spmv(None, x, y, reps=10, fn=lambda: sp.spmv_gather_probe(dA, x, gsum))
        rec["P"], rec["P0"] = P, P0
        per.append(rec)

    launches_per_step = sum(r["P"].info().launches for r in per)
    # ---------------- timed region
    for _ in range(args.warmup):
        for r, x, y in zip(per, xs, ys):
            sp.spmv(r["P"], x, y)
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in per] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    g0.record()
    for k in range(args.steps):
        for m, (r, x, y) in enumerate(zip(per, xs, ys)):
            ev[k][m][0].record()
            sp.spmv(r["P"], x, y)
            ev[k][m][1].record()
    g1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    total_ms = _max_over_ranks(g0.elapsed_time(g1), ws, "cuda")
    kern_ms = [statistics.mean(ev[k][m][0].elapsed_time(ev[k][m][1]) for k in range(args.steps))
               for m in range(len(per))]
    step_bytes = sum(r["min_bytes"] for r in per)
    value = _job_gbs(step_bytes, args.steps, ws, total_ms)

    # ---------------- a secondary figure: the same step with the four
    # independent SpMVs issued on four streams (fork and join by events), so
    # that their kernels overlap at the tails and where one is bound by its
    # gathers of x and another by HBM.  The headline value above stays the
    # sequential step, whose per-kernel times the roofline uses.
    main = torch.cuda.current_stream()
    cstreams = [torch.cuda.Stream() for _ in per]

    def conc_step():
        fork = torch.cuda.Event()
        fork.record(main)
        for r, x, y, st in zip(per, xs, ys, cstreams):
            st.wait_event(fork)
            sp.spmv(r["P"], x, y, stream=st)
        for st in cstreams:
            join = torch.cuda.Event()
            join.record(st)
            main.wait_event(join)
    for _ in range(args.warmup):
        conc_step()
    torch.cuda.synchronize()
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(main)
    for _ in range(args.steps):
        conc_step()
    c1.record(main)
    torch.cuda.synchronize()
    conc_ms = _max_over_ranks(c0.elapsed_time(c1), ws, "cuda")
    concurrent = {"value": round(_job_gbs(step_bytes, args.steps, ws, conc_ms), 2), "unit": "GB/s",
                  "ms_per_step": round(conc_ms / args.steps, 5),
                  "note": "the same step, the four SpMVs on four streams (secondary figure)"}
    # and as one persistent batched launch of the library (every matrix in
    # its prepared sliced layout, launch shapes autotuned, CUDA graph)
    B = sp.spmv_batch_create_sliced([r["P"] for r in per])
    sp.spmv_batch_bind(B, xs, ys)
    sp.spmv_batch_autotune(B)
    for _ in range(args.warmup):
        sp.spmv_batch_run(B, use_graph=True)
    torch.cuda.synchronize()
    c0.record(main)
    for _ in range(args.steps):
        sp.spmv_batch_run(B, use_graph=True)
    c1.record(main)
    torch.cuda.synchronize()
    batch_ms = _max_over_ranks(c0.elapsed_time(c1), ws, "cuda")
    batched = {"value": round(_job_gbs(step_bytes, args.steps, ws, batch_ms), 2), "unit": "GB/s",
               "ms_per_step": round(batch_ms / args.steps, 5),
               "note": "the same step as one persistent batched launch (secondary figure)"}
    B.free()

    # ---------------- end to end through the public API with host buffers:
    # every step uploads each matrix's x from pinned memory, runs its SpMV
    # and downloads y (spmv_host_async, one stream per matrix so that one
    # matrix's copies overlap another's SpMV).  The steps are pipelined: the
    # host waits for the streams once, after the last step, and each matrix
    # has a second prepared object (its own staging buffers) on a second
    # stream, used on alternate steps, so that one step's uploads and
    # downloads overlap the next step's SpMVs.  The same with one object
    # per matrix and a wait after every step is reported beside it, and the
    # bound the host link sets (the step's copies at the link's measured
    # rate, both directions at once).
    hx = [x.cpu().pin_memory() for x in xs]
    hy = [[torch.empty(A.n_rows, dtype=torch.float64).pin_memory() for A in mats] for _ in range(2)]
    streams = [[torch.cuda.Stream() for _ in mats] for _ in range(2)]
    twin = [sp.spmv_prepare(dA, r["choice"]) for dA, r in zip(dev, per)]
    objs = [[r["P"] for r in per], twin]

    def e2e_step(k, wait):
        b = 0 if wait else k % 2
        for P, a, hb, st in zip(objs[b], hx, hy[b], streams[b]):
            sp.spmv_host_async(P, a, hb, stream=st)
        if wait:
            for st in streams[b]:
                st.synchronize()
    for k in range(2):
        e2e_step(k, False)
    torch.cuda.synchronize()
    # three trials of K steps each; the median trial is reported (the host
    # link and host memory are shared with the machine's other GPUs, so a
    # single short trial can catch another job's copies)
    e2e_trials = {False: [], True: []}
    for _ in range(3):
        for wait in (False, True):
            t0 = time.perf_counter()
            for k in range(args.steps):
                e2e_step(k, wait)
            torch.cuda.synchronize()
            e2e_trials[wait].append(time.perf_counter() - t0)
    e2e_s = {w: statistics.median(t) for w, t in e2e_trials.items()}
    for P in twin:
        P.free()
    h2d_b, d2h_b = sum(8 * A.n_cols for A in mats), sum(8 * A.n_rows for A in mats)
    link = _link_gbs(torch, max(h2d_b, d2h_b))
    e2e = {"value": step_bytes * args.steps / e2e_s[False] / 1e9, "unit": "GB/s",
           "h2d_bytes_per_step": h2d_b, "d2h_bytes_per_step": d2h_b,
           "pipelined_steps": True, "prepared_objects_per_matrix": 2,
           "trials": [round(step_bytes * args.steps / t / 1e9, 1) for t in e2e_trials[False]],
           "value_waiting_every_step": step_bytes * args.steps / e2e_s[True] / 1e9,
           "link_gbs": {k: round(v, 1) for k, v in link.items()},
           "link_bound": round(step_bytes / ((h2d_b + d2h_b) / (link["both_directions"] * 1e9)) / 1e9, 1)}

    # ---------------- report
    dom = int(np.argmax(kern_ms))
    achieved = per[dom]["min_bytes"] / (kern_ms[dom] * 1e-3) / 1e9
    plain_total = sum(r["plain_ms"] for r in per)
    sel_total = sum(kern_ms)
    speedups = [r["plain_ms"] / km for r, km in zip(per, kern_ms)]
    matrices = []
    for r, km, s in zip(per, kern_ms, speedups):
        matrices.append({
            "matrix": r["matrix"], "class": r["class"], "variant": r["variant"], "launch": r["launch"],
            "variant_rule": r["variant_rule"], "rule_launch": r["rule_launch"],
            "rule_ms": round(r["rule_ms"], 5), "selected_alone_ms": round(r["selected_alone_ms"], 5),
            "best_variant": r["best_variant"], "ms": round(km, 5),
            "gbs": round(r["min_bytes"] / (km * 1e-3) / 1e9, 1),
            "gflops": round(2 * r["nnz"] / (km * 1e-3) / 1e9, 1),
            "frac_hbm": round(r["min_bytes"] / (km * 1e-3) / 1e9 / peak, 4),
            "plain_gbs": round(r["min_bytes"] / (r["plain_ms"] * 1e-3) / 1e9, 1),
            "speedup_vs_plain": round(s, 3),
            "best_over_selected": (round(km / min(r["variant_ms"].values()), 3)
                                   if r["variant_ms"] else None),
            "features_spmvs": round(r["features_ms"] / r["plain_ms"], 2),
            "profile_spmvs": round(r["profile_select_ms"] / r["plain_ms"], 1),
            "features_selected_spmvs": round(r["features_ms"] / km, 2),
            "profile_selected_spmvs": round(r["profile_select_ms"] / km, 1),
            "prepare_ms": round(r["prepare_ms"], 2),
            "gather_probe_ms": round(r["gather_ms"], 5),
            "hbm_floor_ms": round(r["min_bytes"] / peak / 1e6, 5),
            "variant_ms": r["variant_ms"], "profile": r["profile"]})
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.scale == 0 else WORKLOAD + f" (rows / 2^{args.scale})",
                   "selection": (("learned selector on Table 1 features" +
                                  (", two levels (variant, then SLICED launch configuration)" if sub else ""))
                                 if model is not None else "profiling-based rule (Section 3.2.1)"),
                   "l2": "no flush: every matrix (>= 369 MB) is larger than the 129 MB L2",
                   "parallelism": f"replicas x{ws}"},
        "frac_of_hbm_peak": round(value / peak, 4),
        "gflops": round(2 * sum(r["nnz"] for r in per) * args.steps * ws / (total_ms * 1e-3) / 1e9, 1),
        "plain_csr_gbs": round(step_bytes / (plain_total * 1e-3) / 1e9, 2),
        "speedup_vs_plain_csr": round(plain_total / sel_total, 3),
        "speedup_geomean": round(math.exp(sum(map(math.log, speedups)) / len(speedups)), 3),
        "speedup_geomean_alone": {
            "learned_selector": round(math.exp(sum(math.log(r["plain_ms"] / r["selected_alone_ms"]) for r in per)
                                               / len(per)), 3),
            "profile_rule": round(math.exp(sum(math.log(r["plain_ms"] / r["rule_ms"]) for r in per)
                                           / len(per)), 3),
            "note": "each matrix's choice timed alone, as plain CSR is"},
        "selector_cost_spmvs": {
            "features_and_model": round(sum(r["features_ms"] / r["plain_ms"] for r in per) / len(per), 2),
            "profile_and_rule": round(sum(r["profile_select_ms"] / r["plain_ms"] for r in per) / len(per), 1),
            "unit": "plain-CSR SpMVs of the same matrix, mean over the four",
            "features_and_model_selected": round(sum(r["features_ms"] / km for r, km in zip(per, kern_ms))
                                                 / len(per), 2),
            "profile_and_rule_selected": round(sum(r["profile_select_ms"] / km for r, km in zip(per, kern_ms))
                                               / len(per), 1),
            "unit_selected": "SpMVs of the selected variant of the same matrix, mean over the four"},
        "roofline": {"bound": "hbm", "kernel": f"{per[dom]['variant']} on {per[dom]['matrix']}",
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4),
                     "traffic": _traffic(per[dom]["variant"], per[dom]["matrix"]),
                     "peak_source": f"{peak_kind} HBM copy bandwidth",
                     "gather_probe_ms": round(per[dom]["gather_ms"], 5)},
        "matrices": matrices,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk, "e2e": e2e, "concurrent_streams": concurrent, "batched_launch": batched,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        gbs, sample, rates = cpu_oracle_rate(mats, args.cpu_seconds, 16)
        line["cpu_baseline"] = {"value": round(gbs, 3), "unit": "GB/s", "cores": 1,
                                "kind": "oracle", "sample": sample, "host": _host(),
                                "trials": [round(r, 3) for r in rates]}
        line["cpu_table2"] = cpu_table2_rate(mats)
    for r in per:
        r["P"].free()
        r["P0"].free()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_single(args):
    """One matrix, one variant, a few SpMVs: the command profiled with ncu."""
    import torch
    import paper_1511_02494_gb300 as sp
    import synth
    from paper_1511_02494_gb300.build import build
    build()
    v, _, kv = args.single.partition(":")
    kw = {k: int(val) for k, val in (p.split("=") for p in kv.split(",") if p)}
    make = {"stencil": lambda: synth.stencil_27pt(128), "random": lambda: synth.random_columns(),
            "zipf": lambda: synth.zipf_rows(), "short": lambda: synth.short_rows()}
    A = make[args.matrix]()
    dA = sp.DeviceCSR.from_host(A)
    x = synth.uniform_vector(A.n_cols, 0).cuda()
    y = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
    P = sp.spmv_prepare(dA, sp.make_choice(v, **kw))
    for _ in range(3):
        sp.spmv(P, x, y)
    torch.cuda.synchronize()
    sp.spmv_prepared_status(P)
    print(json.dumps({"single": args.single, "matrix": A.name, "info": P.info().as_dict()}))
    return 0


def _link_gbs(torch, nbytes: int) -> dict:
    """Host link rates (GB/s) of pinned-memory copies of nbytes: each
    direction alone, and both directions at once (aggregate)."""
    n = max(1, nbytes // 8)
    h1 = torch.ones(n, dtype=torch.float64).pin_memory()
    h2 = torch.empty(n, dtype=torch.float64).pin_memory()
    d1 = torch.empty(n, dtype=torch.float64, device="cuda")
    d2 = torch.ones(n, dtype=torch.float64, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def rate(fn, moved, reps=5):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return moved * reps / (time.perf_counter() - t0) / 1e9

    def both():
        with torch.cuda.stream(s1):
            d1.copy_(h1, non_blocking=True)
        with torch.cuda.stream(s2):
            h2.copy_(d2, non_blocking=True)
    return {"h2d": rate(lambda: d1.copy_(h1, non_blocking=True), 8 * n),
            "d2h": rate(lambda: h2.copy_(d2, non_blocking=True), 8 * n),
            "both_directions": rate(both, 16 * n)}


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _time_ms(fn, reps=10, warm=3):
    import torch
    for _ in range(warm):
        fn()
    e0, e1 = _events()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def run_cg(args):
    """Mixed precision: compressed and sliced SpMV throughput with FP32/BF16
    values (FP32 or FP64 accumulation), and CG iterations (300 by default; sliced inner
    and exact SpMV) on the SPD 7-point Laplacian 128^3 (variable
    coefficients) with an FP64, FP32 or BF16 inner SpMV and FP64 residual
    recomputation; errors are against the FP64 GPU solve."""
    import torch
    import paper_1511_02494_gb300 as sp
    import synth
    from paper_1511_02494_gb300.build import build
    build()
    out = {"mode": "mixed_precision", "spmv": [], "cg": []}
    for A in (synth.stencil_27pt(128), synth.random_columns()):
        dA = sp.DeviceCSR.from_host(A)
        x = synth.uniform_vector(A.n_cols, 0).cuda()
        y = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
        yref = torch.empty_like(y)
        P64 = sp.spmv_prepare(dA, sp.make_choice("subwarp"))
        sp.spmv(P64, x, yref)
        for var, name, vt, acc in (
                ("compressed", "f64", sp.VAL_F64, sp.ACC_F64), ("compressed", "f32", sp.VAL_F32, sp.ACC_F32),
                ("compressed", "bf16", sp.VAL_BF16, sp.ACC_F32), ("compressed", "f32_acc64", sp.VAL_F32, sp.ACC_F64),
                ("compressed", "bf16_acc64", sp.VAL_BF16, sp.ACC_F64), ("sliced", "f64", sp.VAL_F64, sp.ACC_F64),
                ("sliced", "f32", sp.VAL_F32, sp.ACC_F32), ("sliced", "bf16", sp.VAL_BF16, sp.ACC_F32),
                ("sliced", "f32_acc64", sp.VAL_F32, sp.ACC_F64), ("sliced", "bf16_acc64", sp.VAL_BF16, sp.ACC_F64)):
            P = sp.spmv_prepare(dA, sp.make_choice(var, value_type=vt, accumulate=acc))
            ms = _time_ms(lambda: sp.spmv(P, x, y))
            sp.spmv(P, x, y)
            scale = torch.linalg.vector_norm(yref, float("inf")).item()
            err = (torch.linalg.vector_norm(y - yref, float("inf")) / scale).item()
            mb = P.info().min_bytes
            out["spmv"].append({"matrix": A.name, "variant": var, "values": name, "ms": round(ms, 5),
                                "min_bytes": mb, "gbs": round(mb / ms / 1e6, 1),
                                "rel_err_vs_f64": err, "wide_rows": P.info().n_wide_rows})
            P.free()
        P64.free()
    A = synth.variable_coeff_laplacian_3d(128, seed=0)
    dA = sp.DeviceCSR.from_host(A)
    b = synth.uniform_vector(A.n_rows, 1).cuda()
    exact = sp.spmv_prepare(dA, sp.make_choice("sliced"))
    iters = args.iters
    xs = {}
    for name, vt, acc, refine in (("f64", None, 0, 0), ("f32", sp.VAL_F32, sp.ACC_F32, 10),
                                  ("bf16", sp.VAL_BF16, sp.ACC_F32, 10),
                                  ("bf16_no_refine", sp.VAL_BF16, sp.ACC_F32, 0),
                                  ("f32_acc64", sp.VAL_F32, sp.ACC_F64, 10),
                                  ("bf16_acc64", sp.VAL_BF16, sp.ACC_F64, 10),
                                  ("bf16_acc64_no_refine", sp.VAL_BF16, sp.ACC_F64, 0)):
        inner = exact if vt is None else sp.spmv_prepare(dA, sp.make_choice("sliced", value_type=vt,
                                                                             accumulate=acc))
        x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
        res = torch.empty(iters + 1, dtype=torch.float64, device="cuda")
        sp.spmv_cg(inner, b, x, iters, refine, A_exact=exact, resid=res, use_graph=True)
        torch.cuda.synchronize()
        e0, e1 = _events()
        x.zero_()
        e0.record()
        sp.spmv_cg(inner, b, x, iters, refine, A_exact=exact, resid=res, use_graph=True)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        r = torch.empty_like(b)
        sp.spmv(exact, x, r)
        true_res = (torch.linalg.vector_norm(b - r) / torch.linalg.vector_norm(b)).item()
        xs[name] = x.clone()
        out["cg"].append({"inner": name, "refine_every": refine, "iters": iters,
                          "ms_total": round(ms, 3), "ms_per_iter": round(ms / iters, 5),
                          "true_rel_residual": true_res,
                          "recursive_rel_residual": (res[-1] / res[0]).item()})
    for rec in out["cg"]:
        d = xs[rec["inner"]] - xs["f64"]
        rec["rel_err_vs_f64_solution"] = (torch.linalg.vector_norm(d) / torch.linalg.vector_norm(xs["f64"])).item()
    out["cg_matrix"] = {"name": A.name, "n_rows": A.n_rows, "nnz": A.nnz}
    print(json.dumps(out), flush=True)
    return 0


def run_coding(args):
    """Column-index forms of SLICED with FP64 values on the four benchmark
    matrices, each in SLICED's automatic layout: 32-bit columns; offsets
    from the row index in 8 or 16 bits where they fit (index_bytes); Table 2's
    delta coding, 8 or 16 bits (index_coding 1, which falls back to panels
    for wide rows); the column-blocked form (index_coding 2).  Time per SpMV
    (CUDA events, mean of 20 after 3 warm-ups), the format's own bytes, and
    whether y equals the 32-bit form's bit for bit (the same DFMA chain)."""
    import torch
    import paper_1511_02494_gb300 as sp
    import synth
    from paper_1511_02494_gb300.build import build
    build()
    out = {"mode": "column_coding", "rows": []}
    for A in synth.four_class_set():
        dA = sp.DeviceCSR.from_host(A)
        x = synth.uniform_vector(A.n_cols, 0).cuda()
        y0 = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
        y = torch.empty_like(y0)
        base = None
        for form, kw in (("int32", {"index_bytes": 4}), ("row_offset", {"index_bytes": 1}),
                         ("delta", {"index_coding": 1}), ("panel", {"index_coding": 2})):
            P = sp.spmv_prepare(dA, sp.make_choice("sliced", **kw))
            info = P.info()
            ms = _time_ms(lambda: sp.spmv(P, x, y), reps=20)
            sp.spmv(P, x, y)
            if base is None:
                base = ms
                y0.copy_(y)
            torch.cuda.synchronize()
            out["rows"].append({"matrix": A.name, "form": form, "index_coding": info.index_coding,
                                "index_bytes": info.index_bytes, "ms": round(ms, 5),
                                "vs_int32": round(base / ms, 3), "format_bytes": info.min_bytes,
                                "csr_gbs": round(A.min_bytes() / (ms * 1e-3) / 1e9, 1),
                                "same_y_as_int32": bool(torch.equal(y, y0))})
            P.free()
    print(json.dumps(out), flush=True)
    return 0


def run_features(args):
    """Feature extraction (Table 1) on the four-class matrices: wall time of
    spmv_features (kernel, readback, host derivation) against the selected
    SpMV, and its bytes: rowptr and colind once."""
    import numpy as np
    import torch
    import paper_1511_02494_gb300 as sp
    import synth
    from paper_1511_02494_gb300.build import build
    build()
    out = {"mode": "features", "matrices": []}
    for A in synth.four_class_set():
        dA = sp.DeviceCSR.from_host(A)
        for _ in range(3):
            sp.spmv_features(dA)
        ts = []
        for _ in range(7):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sp.spmv_features(dA)
            ts.append((time.perf_counter() - t0) * 1e3)
        ms = float(np.median(ts))
        nbytes = 4 * (A.n_rows + 1) + 4 * A.nnz
        P = sp.spmv_prepare(dA, sp.make_choice("sliced"))
        x = synth.uniform_vector(A.n_cols, 0).cuda()
        y = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
        spmv_ms = _time_ms(lambda: sp.spmv(P, x, y))
        out["matrices"].append({"matrix": A.name, "features_ms": round(ms, 4), "bytes": nbytes,
                                "gbs": round(nbytes / ms / 1e6, 1), "sliced_spmv_ms": round(spmv_ms, 4),
                                "features_in_spmvs": round(ms / spmv_ms, 2)})
        P.free()
        del dA
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)
    return 0


def run_batch(args):
    """512 uneven matrices, each with the variant the learned selector picks:
    one launch per matrix with that variant, against one persistent launch
    over all of them (plain, graph, autotuned) with each matrix in the
    persistent form of its variant, and the same with every matrix in the
    sliced layout."""
    import numpy as np
    import torch
    import paper_1511_02494_gb300 as sp
    import synth
    from paper_1511_02494_gb300.build import build
    build()
    mats = synth.batch_matrices(512, seed=0)
    dev = [sp.DeviceCSR.from_host(A) for A in mats]
    xs = [synth.uniform_vector(A.n_cols, i).cuda() for i, A in enumerate(mats)]
    ys = [torch.empty(A.n_rows, dtype=torch.float64, device="cuda") for A in mats]
    total_bytes = sum(A.min_bytes() for A in mats)
    model, sub = _models(sp)
    t0 = time.perf_counter()
    sel = []
    for dA in dev:
        f = sp.spmv_features(dA)
        sel.append(sp.spmv_select_model_refined(f, model, sub) if model is not None
                   else sp.make_choice("subwarp"))
    select_s = time.perf_counter() - t0
    choices = [c.variant for c in sel]
    preps = [sp.spmv_prepare(dA, c, trusted=True) for dA, c in zip(dev, sel)]

    def per_matrix():
        for P, x, y in zip(preps, xs, ys):
            sp.spmv(P, x, y)
    ms_sep = _time_ms(per_matrix, reps=5, warm=2)
    ms_plain = ms_graph = ms_tuned = ms_sliced = tune_s = None
    t = np.zeros(0, np.int32)
    if args.batch_form in ("both", "variant"):
        # one persistent launch, each matrix in the persistent form of its variant
        B = sp.spmv_batch_create_prepared(preps)
        sp.spmv_batch_bind(B, xs, ys)
        ms_plain = _time_ms(lambda: sp.spmv_batch_run(B), reps=10)
        ms_graph = _time_ms(lambda: sp.spmv_batch_run(B, use_graph=True), reps=10)
        t0 = time.perf_counter()
        sp.spmv_batch_autotune(B, reps=3)
        tune_s = time.perf_counter() - t0
        ms_tuned = _time_ms(lambda: sp.spmv_batch_run(B, use_graph=True), reps=10)
        t, _ = sp.spmv_batch_config(B)
    if args.batch_form in ("both", "sliced"):
        # the same with every matrix in the sliced layout
        Bs = sp.spmv_batch_create_sliced(preps)
        sp.spmv_batch_bind(Bs, xs, ys)
        sp.spmv_batch_autotune(Bs, reps=3)
        ms_sliced = _time_ms(lambda: sp.spmv_batch_run(Bs, use_graph=True), reps=10)

    def r4(v):
        return None if v is None else round(v, 4)

    def gbs(v):
        return None if v is None else round(total_bytes / v / 1e6, 1)
    out = {"mode": "batched", "matrices": len(mats), "nnz": int(sum(A.nnz for A in mats)),
           "rows_range": [min(A.n_rows for A in mats), max(A.n_rows for A in mats)],
           "min_bytes": total_bytes,
           "selection": (("learned selector" + (", two levels" if sub else "")) if model is not None
                         else "sub-warp default"),
           "selection_s": round(select_s, 3),
           "variant_counts": {sp.VARIANTS[v]: int(c) for v, c in
                              zip(*np.unique(np.array(choices), return_counts=True))},
           "ms_one_launch_per_matrix": round(ms_sep, 4),
           "ms_persistent": r4(ms_plain), "ms_persistent_graph": r4(ms_graph),
           "ms_persistent_graph_autotuned": r4(ms_tuned),
           "autotune_s": None if tune_s is None else round(tune_s, 2),
           "gbs_one_launch_per_matrix": round(total_bytes / ms_sep / 1e6, 1),
           "gbs_persistent_graph_autotuned": gbs(ms_tuned),
           "ms_persistent_sliced_graph_autotuned": r4(ms_sliced),
           "gbs_persistent_sliced_graph_autotuned": gbs(ms_sliced),
           "autotuned_lanes_per_row_counts": {int(k): int(c) for k, c in
                                              zip(*np.unique(t, return_counts=True))}}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=0, help="shrink rows by 2^scale (not for records)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variant-sweep", action="store_true",
                    help="skip timing every variant per matrix (best-variant fields become null)")
    ap.add_argument("--single", default=None,
                    help="VARIANT[:k=v,...]: run only this variant on --matrix (for ncu)")
    ap.add_argument("--matrix", default="stencil", choices=["stencil", "random", "zipf", "short"])
    ap.add_argument("--cg", action="store_true", help="mixed-precision SpMV and CG report")
    ap.add_argument("--iters", type=int, default=300, help="CG iterations of --cg")
    ap.add_argument("--batch", action="store_true", help="batched persistent SpMV report")
    ap.add_argument("--batch-form", default="both", choices=["both", "variant", "sliced"],
                    help="--batch: which persistent form(s) to run")
    ap.add_argument("--features", action="store_true", help="feature extraction report")
    ap.add_argument("--coding", action="store_true", help="column-index forms of SLICED report")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.single:
        return run_single(args)
    if args.cg:
        return run_cg(args)
    if args.features:
        return run_features(args)
    if args.coding:
        return run_coding(args)
    if args.batch:
        return run_batch(args)
    return run_reference(args) if args.impl == "reference" else run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
