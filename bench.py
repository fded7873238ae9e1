"""Benchmark of the batched Fast DCT+ forward transform on GB300.

Headline workload (one "step" = one forward pass over the whole batch):
mixed-size rows, 2^20 rows with n drawn uniformly from {4, 8, 16, 32, 64},
integer Laplace(12) residuals clipped to [-255, 255] in FP32, four rank-one
updates per size (self-loop at vertex 0 with rho in {0.5, 1, 2}, central-edge
weight change rho = -0.5), all 20 (size, update) segments in one persistent
launch replayed from a CUDA graph. A second line item times n = 1024 signals
(batch 4096, dense random unit v, rho in {-0.3, 2.0}).

Run:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "transform GSamples/s + %roofline at n=64/1024 vs dense-GFT GEMM, same GPU, FP32 err"
WORKLOAD = ("mixed-size forward: 2^20 rows, n uniform in {4,8,16,32,64}, rint(Laplace(0,12)) "
            "clipped to [-255,255] FP32, 4 rank-one updates per size (self-loop at vertex 0, "
            "rho in {0.5,1,2}; edge (n/2-1,n/2), rho=-0.5), one persistent launch per step from a "
            "CUDA graph")
L2_FLUSH_BYTES = 256 << 20


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


# TF32 dense tensor rate relative to BF16 (nominal 1.1 vs 2.25 PFLOP/s per GPU): the peak of
# the split-TF32 contractions is the measured BF16 cuBLAS figure times this ratio.
TF32_PER_BF16 = 1.1 / 2.25
# FP64 on the CUDA cores (nominal, no measured figure): 1.25 TFLOP/s
FP64_NOMINAL_TFLOPS = 1.25
TENSOR_KERNELS = ("k_gemm_tc", "k_small_tc")
FP64_ALU_KERNELS = ("k_nfst_fast", "k_nfst_route")  # the paper's route: FP64 arithmetic on CUDA cores


def trace_kernels(pkg, torch, stream, step, flush, reps=3):
    """Per-launch device time of one step, from the library's kernel trace (CUDA events after
    every launch on the step's stream, outside graph capture, L2 flushed before each step).
    Returns one record per launch position: name, median ms over reps, bytes, flops."""
    sh = stream.cuda_stream
    runs = []
    for _ in range(reps):
        with torch.cuda.stream(stream):
            flush()
        pkg.dctplus_trace_begin(sh)
        step()
        runs.append(pkg.dctplus_trace_end(sh))
    out = []
    for i, rec in enumerate(runs[0]):
        ms = float(np.median([r[i][1] for r in runs if len(r) > i]))
        out.append({"kernel": rec[0], "ms": ms, "bytes": rec[2], "flops": rec[3]})
    return out


def roofline_of(recs, hbm_peak, bf16_peak, peak_src):
    """Roofline object of the dominant kernel (largest summed time over the step's launches of
    that kernel): tensor-bound for the tensor-core GEMMs (split-TF32 peak), FP64-ALU bound for
    the paper's trigonometric route (nominal FP64 rate), HBM otherwise."""
    by = {}
    for r in recs:
        e = by.setdefault(r["kernel"], {"ms": 0.0, "bytes": 0.0, "flops": 0.0, "launches": 0})
        e["ms"] += r["ms"]
        e["bytes"] += r["bytes"]
        e["flops"] += r["flops"]
        e["launches"] += 1
    total = sum(e["ms"] for e in by.values())
    name, e = max(by.items(), key=lambda kv: kv[1]["ms"])
    per_launch_ms = e["ms"] / e["launches"]
    if name in TENSOR_KERNELS and name != "k_small_tc":
        peak = bf16_peak * TF32_PER_BF16
        achieved = e["flops"] / e["launches"] / (per_launch_ms * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "peak_source": f"{peak_src} bf16_tflops x {TF32_PER_BF16:.4f} (TF32/BF16 nominal "
                               "1.1/2.25 PFLOP/s): split-TF32 products counted as executed",
                "algorithmic_flops_per_launch": e["flops"] / e["launches"]}
    elif name in FP64_ALU_KERNELS:
        achieved = e["flops"] / e["launches"] / (per_launch_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_NOMINAL_TFLOPS,
                "peak_source": "nominal FP64 CUDA-core rate (no measured FP64 figure)",
                "algorithmic_flops_per_launch": e["flops"] / e["launches"]}
    else:
        achieved = e["bytes"] / e["launches"] / (per_launch_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "peak_source": f"{peak_src} hbm_gbs (burst copy)",
                "algorithmic_bytes_per_launch": e["bytes"] / e["launches"]}
    roof.update({"kernel": name, "kernel_ms": per_launch_ms, "launches_of_kernel": e["launches"],
                 "share_of_step": e["ms"] / total if total > 0 else None, "traffic": None,
                 "stages": [{"kernel": r["kernel"], "ms": round(r["ms"], 5)} for r in recs]})
    return roof


_ORACLE_PLANS = {}


def oracle_plan(n, v, rho, roots=None):
    """The oracle's plan for (n, v, rho[, sampled roots]), built once per bench run (its
    secular solve is O(n^2) per root set in FP64 on the host)."""
    from oracle import cauchy
    key = (n, float(rho), np.asarray(v, dtype=np.float64).tobytes(),
           None if roots is None else tuple(int(r) for r in roots))
    if key not in _ORACLE_PLANS:
        _ORACLE_PLANS[key] = (cauchy.make_plan(n, v, rho) if roots is None
                              else cauchy.make_plan(n, v, rho, roots=roots))
    return _ORACLE_PLANS[key]


def oracle_rate(fn, samples_per_call, sample, budget_s=1.0):
    """The FP64 oracle timed as it stands on the host cores: fn() repeated for about budget_s
    seconds (plan creation excluded), as input samples per second."""
    calls = 0
    t0 = time.perf_counter()
    while True:
        fn()
        calls += 1
        elapsed = time.perf_counter() - t0
        if elapsed >= budget_s:
            break
    return {"value": calls * samples_per_call / elapsed / 1e9, "unit": "GSamples/s",
            "cores": len(os.sched_getaffinity(0)), "kind": "oracle", "sample": sample}


def oracle_error(n, v, rho, x, y, sig_rows=8, root_sample=None, seed=7):
    """FP32 output against the FP64 oracle (Cauchy formula) on a sampled subset of signals: all
    rows up to n = 4096, else about 40 sampled secular-root rows. Errors relative to the
    signal's norm (max) and normwise over the compared rows."""
    from oracle import cauchy
    rng = np.random.default_rng(seed)
    sig = np.sort(rng.choice(x.shape[0], min(sig_rows, x.shape[0]), replace=False))
    xs = x[sig].astype(np.float64)
    if n <= 4096 and root_sample is None:
        op = oracle_plan(n, v, rho)
        cols = np.arange(n)
    else:
        probe = oracle_plan(n, v, rho, roots=[])
        K = int(probe.row_kind.sum())
        roots = np.unique(np.concatenate([rng.choice(K, min(K, root_sample or 36), replace=False),
                                          [0, K - 1]]))
        op = oracle_plan(n, v, rho, roots=roots)
        cols = np.nonzero((op.row_kind == 1) & np.isin(op.row_index, roots))[0]
    ref = cauchy.transform(op, xs, rows=cols)
    got = y[sig][:, cols].astype(np.float64)
    diff = got - ref
    nrm = np.linalg.norm(xs, axis=1)
    rel = np.linalg.norm(diff, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-300)
    return {"max_abs": float(np.abs(diff).max()),
            "max_abs_rel_to_signal_norm": float((np.abs(diff).max(axis=1) / nrm).max()),
            "normwise_rel_max": float(rel.max()),
            "snr_db_mean": float(np.mean(-20 * np.log10(np.maximum(rel, 1e-300)))),
            "sample": f"{len(sig)} signals x {len(cols)} coefficients"
                      + ("" if len(cols) == n else " (sampled secular-root rows)")}


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, world: int) -> float:
    """Largest value over the ranks (a step counts when the slowest replica is done)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(samples_per_rank: float, seconds_max: float, world: int) -> float:
    """GSamples/s of the whole job: every rank runs its own replica of the workload."""
    return world * samples_per_rank / seconds_max / 1e9


def make_mixed(pkg):
    from synthetic import mixed_size_workload
    wl = mixed_size_workload()
    plans, index = [], {}
    for n, ups in wl.updates.items():
        for u, (v, rho) in enumerate(ups):
            index[(n, u)] = len(plans)
            plans.append(pkg.Plan(n, v, rho))
    seg = np.array([[index[(s.n, s.update)], s.offset, s.rows] for s in wl.segments], dtype=np.int64)
    return wl, plans, seg


def profiled_traffic():
    """DRAM bytes (read + write) per launch of the headline kernel from its committed ncu
    summary, or None when the kernel's sources changed since that capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "k_small_tc_mixed_2p20.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    fields = dict(line.strip().split(": ", 1) for line in text.splitlines()
                  if line.strip().startswith(("source_sha256: ", "traffic_bytes_per_launch: ")))
    h = hashlib.sha256()
    for f in ("small_tc.cu", "tc_ptx.cuh"):
        with open(os.path.join(ROOT, "paper_2409_08970_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if fields.get("source_sha256") != h.hexdigest() or "traffic_bytes_per_launch" not in fields:
        return None
    return int(fields["traffic_bytes_per_launch"])


def time_graph(fn, stream, steps, warmup, flush):
    """Capture fn() in a CUDA graph; time `steps` replays with events, flushing L2 between."""
    import torch
    fn()  # first call uploads tables / allocates scratch outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            fn()
    torch.cuda.synchronize()
    for _ in range(warmup):
        flush()
        g.replay()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    with torch.cuda.stream(stream):
        for e0, e1 in evs:
            flush()
            e0.record(stream)
            g.replay()
            e1.record(stream)
    torch.cuda.synchronize()
    return [e0.elapsed_time(e1) for e0, e1 in evs], g


def run_ours(args):
    import torch
    import paper_2409_08970_gb300 as pkg
    from paper_2409_08970_gb300 import build as _build
    rank, world, local = dist_setup()
    if rank == 0:
        _build.build()
    barrier(world)
    hbm_peak, bf16_peak, peak_src = load_peaks()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream()
    flush_buf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def flush():
        flush_buf.fill_(1.0)

    wl, plans, seg = make_mixed(pkg)
    group = pkg.Group(plans)
    x = torch.tensor(wl.x, device=dev)
    y = torch.empty_like(x)
    samples = wl.total_samples
    sh = stream.cuda_stream

    def step():
        pkg.dctplus_execute_group(group.handle, x.data_ptr(), y.data_ptr(), seg, sh)

    lc0 = pkg.dctplus_launch_count()
    step()
    torch.cuda.synchronize()
    launches_per_step = pkg.dctplus_launch_count() - lc0

    clocks = ClockSampler(torch.cuda.current_device())
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    times, graph = time_graph(step, stream, args.steps, args.warmup, flush)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    t_ms = float(np.mean(times))
    t_ms_max = max_over_ranks(t_ms, world)
    value = whole_job_rate(samples, t_ms_max * 1e-3, world)

    # one step is one launch of the tensor-core kernel, so the step's event
    # time is that kernel's duration
    tk_ms = t_ms
    algo_bytes = 8.0 * samples  # read x + write y, FP32
    achieved = algo_bytes / (tk_ms * 1e-3) / 1e9

    # end to end through the host-buffer C entry point (pinned host memory)
    xh = torch.empty(x.numel(), dtype=torch.float32, pin_memory=True)
    xh.copy_(torch.from_numpy(wl.x))
    yh = torch.empty(x.numel(), dtype=torch.float32, pin_memory=True)
    xh_np, yh_np = xh.numpy(), yh.numpy()

    def e2e_step():
        pkg.dctplus_execute_group_host(group.handle, xh_np.ctypes.data, yh_np.ctypes.data,
                                       xh_np.size, seg, sh)

    for _ in range(max(1, args.warmup)):
        e2e_step()
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    t_e2e = (time.perf_counter() - t0) / args.steps
    t_e2e = max_over_ranks(t_e2e, world)
    e2e = {"value": whole_job_rate(samples, t_e2e, world), "unit": "GSamples/s",
           "h2d_bytes_per_step": int(4 * samples), "d2h_bytes_per_step": int(4 * samples),
           "ms_per_step": t_e2e * 1e3}

    extra = {}
    if not args.no_extra and rank == 0:
        D, H, G, R = pkg.CAUCHY_DENSE, pkg.CAUCHY_HIER, pkg.CAUCHY_DENSE_GFT, pkg.CAUCHY_NFST
        peaks = (hbm_peak, bf16_peak, peak_src)
        errs = not args.no_cpu
        extra["fp64_n64"] = bench_fp64_n64(pkg, torch, dev, stream, args, flush, peaks)
        HL, HT = (H, 1), (H, 2)
        extra["n1024"] = bench_large(pkg, torch, dev, stream, args, flush, peaks, 1024, 4096,
                                     [HL, HT, D, G, R], errs)
        if not args.quick:
            extra["n256"] = bench_large(pkg, torch, dev, stream, args, flush, peaks, 256, 4096,
                                        [HL, HT, D, G, R], errs)
            extra["n4096"] = bench_large(pkg, torch, dev, stream, args, flush, peaks, 4096, 4096,
                                         [HL, HT, D, G, R], errs)
            extra["n16384"] = bench_large(pkg, torch, dev, stream, args, flush, peaks, 16384, 512, [HL, HT], errs)
        extra["pruned_n512"] = bench_pruned(pkg, torch, dev, stream, args, flush, peaks)
        extra["backward_n1024"] = bench_backward(pkg, torch, dev, stream, args, flush, peaks)
        extra["dense_gft_cublas_fp32"] = bench_dense_gft(pkg, torch, dev, stream, args, flush, wl,
                                                         plans, seg)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(wl, y.cpu().numpy())

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GSamples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "rows": int(wl.total_rows), "samples": int(samples),
                       "segments": int(seg.shape[0]), "l2": "flushed (256 MiB write) between timed steps",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": profiled_traffic(),
                         "traffic_unit": "bytes per launch (ncu dram read + write)",
                         "peak_source": f"{peak_src} hbm_gbs (burst copy)",
                         "kernel": "k_small_tc" if launches_per_step == 1 else "k_small_tc + k_small_simt",
                         "kernel_ms": tk_ms, "launches_per_step": launches_per_step,
                         "algorithmic_bytes_per_launch": algo_bytes},
            "e2e": e2e,
            "gpu_launches": int(launches_per_step * args.steps),
            "clocks": clk,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu["baseline"]
            line["fp32_err_vs_fp64_oracle"] = cpu["err"]
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


MODE_NAMES = {1: "dense", 2: "hierarchical", 3: "cuda_core", 4: "dense_gft_baseline",
              5: "nfst_route_fp64"}


def bench_large(pkg, torch, dev, stream, args, flush, peaks, n, batch, modes, errors=True):
    """Large-n forward: batch N(0,1) signals, dense unit v (seed 1), rho in {-0.3, 2.0};
    one step = both plans over the batch. Modes are timed one after another. Per mode: the
    step rate, the dominant kernel's roofline (kernel trace), the plan time and the FP32 error
    against the FP64 oracle on sampled signals."""
    from synthetic import normal_signals, random_unit_v
    hbm_peak, bf16_peak, peak_src = peaks
    v = random_unit_v(n)
    xh = normal_signals(batch, n, seed=0)
    x = torch.tensor(xh, dtype=torch.float32, device=dev)
    rhos = (-0.3, 2.0)
    y2 = torch.empty((batch, len(rhos) * n), dtype=torch.float32, device=dev)
    ys = [y2[:, k * n:(k + 1) * n] for k in range(len(rhos))]
    sh = stream.cuda_stream
    samples = 2 * batch * n
    out = {"workload": f"n={n}, batch {batch}, x~N(0,1), dense unit v (seed 1), rho in {{-0.3, 2.0}}; "
                       "one step = both plans over the batch in one dctplus_execute_multi call (the "
                       "hierarchical and dense modes share the DCT-II, the hierarchical mode also the far "
                       "field of the common v; the others run plan by plan)"}
    for mode in modes:
        mode, far = mode if isinstance(mode, tuple) else (mode, 0)
        try:
            t0 = time.perf_counter()
            plans = [pkg.Plan(n, v, rho, cauchy_mode=mode, far_field=far) for rho in rhos]
            plan_ms = (time.perf_counter() - t0) * 1e3 / len(rhos)
        except pkg.DctPlusError:
            continue

        def step():
            pkg.dctplus_execute_multi([p.handle for p in plans], x.data_ptr(), n, y2.data_ptr(),
                                      len(rhos) * n, batch, sh)

        lc = pkg.dctplus_launch_count()
        step()
        torch.cuda.synchronize()
        launches = pkg.dctplus_launch_count() - lc
        times, _ = time_graph(step, stream, args.steps, args.warmup, flush)
        t_ms = float(np.mean(times))
        recs = trace_kernels(pkg, torch, stream, step, flush)
        entry = {"value": samples / (t_ms * 1e-3) / 1e9, "unit": "GSamples/s", "ms_per_step": t_ms,
                 "launches_per_step": launches,
                 "shared_dct": plans[0].cauchy_mode in (pkg.CAUCHY_HIER, pkg.CAUCHY_DENSE),
                 "hbm_frac_of_measured": 8.0 * samples / (t_ms * 1e-3) / 1e9 / hbm_peak,
                 "plan_ms": plan_ms,
                 "roofline": roofline_of(recs, hbm_peak, bf16_peak, peak_src)}
        if errors:
            step()
            torch.cuda.synchronize()
            errs = [oracle_error(n, v, rho, xh, y.cpu().numpy(),
                                 root_sample=36 if n > 4096 else None) for rho, y in zip(rhos, ys)]
            entry["fp32_err_vs_fp64_oracle"] = {
                k: max(e[k] for e in errs) for k in ("max_abs", "max_abs_rel_to_signal_norm",
                                                    "normwise_rel_max")}
            entry["fp32_err_vs_fp64_oracle"]["snr_db_mean"] = float(np.mean([e["snr_db_mean"] for e in errs]))
            entry["fp32_err_vs_fp64_oracle"]["sample"] = errs[0]["sample"] + " per plan"
        name = MODE_NAMES.get(plans[0].cauchy_mode, str(mode))
        if plans[0].cauchy_mode == pkg.CAUCHY_HIER:
            name += {1: "_leaf_level", 2: "_tree"}.get(plans[0].far_field, "")
        out[name] = entry
        for p in plans:
            p.close()
    # one update per step (rho = 2.0, dctplus_execute): nothing shared between updates
    single = {}
    for mode, far in ((pkg.CAUCHY_HIER, 1), (pkg.CAUCHY_DENSE_GFT, 0)):
        try:
            p1 = pkg.Plan(n, v, 2.0, cauchy_mode=mode, far_field=far)
        except pkg.DctPlusError:
            continue

        def step1():
            pkg.dctplus_execute(p1.handle, pkg.F32, x.data_ptr(), n, y2.data_ptr(), 2 * n, batch, sh)

        t1 = float(np.mean(time_graph(step1, stream, args.steps, args.warmup, flush)[0]))
        name = MODE_NAMES.get(p1.cauchy_mode, str(mode))
        if p1.cauchy_mode == pkg.CAUCHY_HIER:
            name += {1: "_leaf_level", 2: "_tree"}.get(p1.far_field, "")
        single[name] = {"value": batch * n / (t1 * 1e-3) / 1e9, "unit": "GSamples/s", "ms_per_step": t1}
        p1.close()
    if single:
        out["one_update_per_step"] = single
    if errors and n <= 4096:  # the oracle beside it (rho = 2.0; all coefficients of k signals)
        from oracle import cauchy
        op = oracle_plan(n, v, 2.0)
        k = max(4, min(256, (1 << 26) // (n * n)))
        xs = xh[:k].astype(np.float64)
        out["cpu_oracle"] = oracle_rate(lambda: cauchy.transform(op, xs), k * n,
                                        f"{k} signals, all {n} coefficients, one plan (rho = 2.0)")
    if n > 64:  # what the autotuner measures and would pick for this n and batch (rho = 2.0)
        t = pkg.dctplus_autotune(n, v, 2.0, batch, None, sh)
        out["autotune"] = {"choice": {1: "dense", 2: "hierarchical", 3: "cuda_core"}.get(t["cauchy_mode"]),
                           "far_field": t["far_field"], "ms_per_call": t["ms"],
                           "note": "per call of one plan over the batch, not L2-flushed"}
    return out


def bench_fp64_n64(pkg, torch, dev, stream, args, flush, peaks):
    """FP64 forward, n = 64, unit self-loop at vertex 0 (v = e_0, rho = 1), 1024 N(0,1)
    signals (seed 0): the FP64 configuration, with its error against the FP64 oracle."""
    from oracle import cauchy
    from synthetic import normal_signals, self_loop_v
    hbm_peak, bf16_peak, peak_src = peaks
    n, batch = 64, 1024
    v = self_loop_v(n, 0)
    xh = normal_signals(batch, n, seed=0)
    x = torch.tensor(xh, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    sh = stream.cuda_stream
    t0 = time.perf_counter()
    plan = pkg.Plan(n, v, 1.0)
    plan_ms = (time.perf_counter() - t0) * 1e3

    def step():
        pkg.dctplus_execute(plan.handle, pkg.F64, x.data_ptr(), n, y.data_ptr(), n, batch, sh)

    times, _ = time_graph(step, stream, args.steps, args.warmup, flush)
    t_ms = float(np.mean(times))
    recs = trace_kernels(pkg, torch, stream, step, flush)
    step()
    torch.cuda.synchronize()
    op = cauchy.make_plan(n, v, 1.0)
    ref = cauchy.transform(op, xh)
    got = y.cpu().numpy()
    rel = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    cpu = oracle_rate(lambda: cauchy.transform(op, xh), batch * n, f"the whole batch ({batch} signals)")
    k = recs[0]
    achieved = k["flops"] / (k["ms"] * 1e-3) / 1e12
    plan.close()
    return {"workload": "FP64, n=64, self-loop weight 1 at vertex 0 (v=e_0), 1024 signals x~N(0,1) "
                        "(seed 0)",
            "value": batch * n / (t_ms * 1e-3) / 1e9, "unit": "GSamples/s", "ms_per_step": t_ms,
            "dtype": "f64", "plan_ms": plan_ms,
            "err_vs_fp64_oracle": {"max_abs": float(np.abs(got - ref).max()),
                                   "normwise_rel_max": float(rel.max())},
            "cpu_oracle": cpu,
            "roofline": {"bound": "alu", "kernel": k["kernel"], "kernel_ms": k["ms"],
                         "achieved": achieved, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_NOMINAL_TFLOPS,
                         "peak_source": "nominal FP64 CUDA-core rate (no measured FP64 figure)",
                         "algorithmic_flops_per_launch": k["flops"],
                         "note": "1024 signals: a few microseconds of work, launch-latency bound"}}


def bench_pruned(pkg, torch, dev, stream, args, flush, peaks, n=512, batch=16384, m_out=128):
    """Progressive multi-transform with pruning (Theorem 3.4): one DCT-II per signal shared by
    K = 8 self-loop updates at vertex 0 (rho = 0.25 .. 2.0), the first m_out coefficients of
    each; exact (c_p = n) and truncated (c_p = m_out), against 8 independent full transforms."""
    from oracle import cauchy
    from synthetic import normal_signals, self_loop_v
    hbm_peak, bf16_peak, peak_src = peaks
    rhos = [0.25 * (k + 1) for k in range(8)]
    t0 = time.perf_counter()
    plans = [pkg.Plan(n, self_loop_v(n, 0), r) for r in rhos]
    plan_ms = (time.perf_counter() - t0) * 1e3 / len(rhos)
    xh = normal_signals(batch, n, seed=0)
    x = torch.tensor(xh, dtype=torch.float32, device=dev)
    sh = stream.cuda_stream
    samples = batch * n
    width = len(plans) * m_out
    y = torch.empty(batch, width, dtype=torch.float32, device=dev)
    ys = [torch.empty_like(x) for _ in plans]
    out = {"workload": f"n={n}, batch {batch}, K=8 self-loop updates at vertex 0 (rho 0.25..2.0), "
                       f"first {m_out} coefficients of each; samples = input samples",
           "plan_ms": plan_ms}
    rng = np.random.default_rng(7)
    sig = np.sort(rng.choice(batch, 8, replace=False))
    ops = [cauchy.make_plan(n, self_loop_v(n, 0), r) for r in rhos]

    def timed(step, bytes_per_step):
        lc = pkg.dctplus_launch_count()
        step()
        torch.cuda.synchronize()
        launches = pkg.dctplus_launch_count() - lc
        times, _ = time_graph(step, stream, args.steps, args.warmup, flush)
        t_ms = float(np.mean(times))
        recs = trace_kernels(pkg, torch, stream, step, flush)
        return {"value": samples / (t_ms * 1e-3) / 1e9, "unit": "GSamples/s", "ms_per_step": t_ms,
                "launches_per_step": launches,
                "hbm_frac_of_measured": bytes_per_step / (t_ms * 1e-3) / 1e9 / hbm_peak,
                "roofline": roofline_of(recs, hbm_peak, bf16_peak, peak_src)}

    handles = [p.handle for p in plans]
    algo_bytes = 4.0 * batch * (n + width)
    for c_p, name in ((n, "pruned_exact"), (m_out, "pruned_truncated_cp")):
        def step(c_p=c_p):
            pkg.dctplus_execute_pruned(handles, x.data_ptr(), n, y.data_ptr(), width, batch, m_out,
                                       c_p, sh)
        out[name] = timed(step, algo_bytes)
        step()
        torch.cuda.synchronize()
        got = y.cpu().numpy()[sig].astype(np.float64)
        err, bound_ok = 0.0, True
        for k, op in enumerate(ops):
            part = got[:, k * m_out:(k + 1) * m_out]
            if c_p == n:  # exact first m_out coefficients
                ref = cauchy.transform(op, xh[sig], rows=np.arange(m_out))
            else:  # Theorem 3.4's truncated block
                ref = cauchy.pruned_transform(op, xh[sig], m_out, c_p)
            err = max(err, float((np.abs(part - ref).max(axis=1) / np.linalg.norm(xh[sig], axis=1)).max()))
        out[name]["fp32_err_vs_fp64_oracle"] = {
            "max_abs_rel_to_signal_norm": err,
            "sample": f"{len(sig)} signals x {m_out} coefficients x {len(ops)} updates"
                      + ("" if c_p == n else "; against the oracle's Theorem 3.4 truncated block")}
        xs = xh[sig].astype(np.float64)
        if c_p == n:
            fn = lambda: [cauchy.transform(op, xs, rows=np.arange(m_out)) for op in ops]
        else:
            fn = lambda: [cauchy.pruned_transform(op, xs, m_out, c_p) for op in ops]
        out[name]["cpu_oracle"] = oracle_rate(fn, len(sig) * n,
                                              f"{len(sig)} signals, {len(ops)} updates, {m_out} coefficients each")

    def full():
        for p, yy in zip(plans, ys):
            pkg.dctplus_execute(p.handle, pkg.F32, x.data_ptr(), n, yy.data_ptr(), n, batch, sh)
    out["eight_full_transforms"] = timed(full, 8.0 * 8 * batch * n)
    for p in plans:
        p.close()
    return out


def bench_backward(pkg, torch, dev, stream, args, flush, peaks, n=1024, batch=8192):
    """Differentiable transform: n = 1024, batch 8192, loss = sum of squared coefficients
    512..1023, dense unit v (seed 1), rho = 2.0. One step = forward + backward to x, rho and v
    (the loss gradient 2 y on the upper half is formed on the device by torch, not timed as
    transform work but inside the step)."""
    from oracle import cauchy, gradient
    from synthetic import normal_signals, random_unit_v
    hbm_peak, bf16_peak, peak_src = peaks
    v = random_unit_v(n)
    t0 = time.perf_counter()
    plan = pkg.Plan(n, v, 2.0)
    plan_ms = (time.perf_counter() - t0) * 1e3
    xh = normal_signals(batch, n, seed=0)
    x = torch.tensor(xh, dtype=torch.float32, device=dev)
    y = torch.empty_like(x)
    g = torch.zeros_like(x)
    gx = torch.empty_like(x)
    g_rho = torch.empty((), dtype=torch.float64, device=dev)
    g_v = torch.empty(n, dtype=torch.float64, device=dev)
    sh = stream.cuda_stream
    samples = batch * n

    def step():
        pkg.dctplus_execute(plan.handle, pkg.F32, x.data_ptr(), n, y.data_ptr(), n, batch, sh)
        with torch.cuda.stream(stream):
            torch.mul(y[:, n // 2:], 2.0, out=g[:, n // 2:])
        pkg.dctplus_backward(plan.handle, g.data_ptr(), n, y.data_ptr(), n, gx.data_ptr(), n,
                             g_rho.data_ptr(), g_v.data_ptr(), batch, sh)

    lc = pkg.dctplus_launch_count()
    step()
    torch.cuda.synchronize()
    launches = pkg.dctplus_launch_count() - lc
    times, _ = time_graph(step, stream, args.steps, args.warmup, flush)
    t_ms = float(np.mean(times))
    recs = trace_kernels(pkg, torch, stream, step, flush)
    step()
    torch.cuda.synchronize()
    op = cauchy.make_plan(n, v, 2.0)
    gh = g.double().cpu().numpy()
    rng = np.random.default_rng(7)
    sig = np.sort(rng.choice(batch, 8, replace=False))
    ref_x = gradient.backward_x(op, gh[sig])
    gxh = gx.double().cpu().numpy()[sig]
    r_rho, r_v = gradient.parameter_gradients(op, xh, gh)
    err = {"gx_normwise_rel_max": float((np.linalg.norm(gxh - ref_x, axis=1)
                                         / np.linalg.norm(ref_x, axis=1)).max()),
           "grad_rho_rel": abs(float(g_rho.item()) - r_rho) / abs(r_rho),
           "grad_v_rel": float(np.linalg.norm(g_v.cpu().numpy() - r_v) / np.linalg.norm(r_v)),
           "sample": "gx on 8 signals; grad_rho and grad_v over the whole batch (the oracle's "
                     "gradients for the same upstream g)"}
    xs, gs = xh[:64], gh[:64]
    cpu = oracle_rate(lambda: (cauchy.transform(op, xs), gradient.backward_x(op, gs),
                               gradient.parameter_gradients(op, xs, gs)), 64 * n,
                      "64 signals: forward, then the gradients to x, rho and v")
    plan.close()
    return {"workload": f"n={n}, batch {batch}, loss = sum y[:, {n // 2}:]^2, dense unit v (seed 1), "
                        "rho = 2.0; forward + backward to x, rho, v",
            "value": samples / (t_ms * 1e-3) / 1e9, "unit": "GSamples/s (forward + backward)",
            "ms_per_step": t_ms, "launches_per_step": launches, "plan_ms": plan_ms,
            "roofline": roofline_of(recs, hbm_peak, bf16_peak, peak_src),
            "fp32_err_vs_fp64_oracle": err, "cpu_oracle": cpu}


def bench_dense_gft(pkg, torch, dev, stream, args, flush, wl, plans, seg):
    """Non-product reference point: cuBLAS FP32 GEMM against the dense X^T per segment.

    X^T comes from this library's FP64 transform of the identity (rows of I).
    """
    torch.backends.cuda.matmul.allow_tf32 = False
    mats = []
    for p in plans:
        eye = torch.eye(p.n, dtype=torch.float64, device=dev)
        mats.append(p.forward(eye).t().contiguous().float())  # X^T
    x = torch.tensor(wl.x, device=dev)
    y = torch.empty_like(x)
    views = []
    for pi, off, rows in seg:
        n = plans[pi].n
        views.append((x[off:off + rows * n].view(rows, n), y[off:off + rows * n].view(rows, n),
                      mats[pi].t()))

    def step():
        for xs, ys, m in views:
            torch.matmul(xs, m, out=ys)

    with torch.cuda.stream(stream):
        times, _ = time_graph(step, stream, args.steps, args.warmup, flush)
    t_ms = float(np.mean(times))
    return {"value": wl.total_samples / (t_ms * 1e-3) / 1e9, "unit": "GSamples/s",
            "ms_per_step": t_ms, "kind": "cuBLAS SGEMM per segment (FP32, no TF32), same workload"}


def cpu_baseline(wl, y_gpu):
    """The FP64 oracle (Cauchy formula, O2) as it stands, on the host cores."""
    from oracle import cauchy
    plans = {(n, u): cauchy.make_plan(n, v, rho) for n, ups in wl.updates.items()
             for u, (v, rho) in enumerate(ups)}
    t0 = time.perf_counter()
    outs = []
    for s in wl.segments:
        xs = wl.x[s.offset:s.offset + s.rows * s.n].astype(np.float64).reshape(s.rows, s.n)
        outs.append(cauchy.transform(plans[(s.n, s.update)], xs))
    dt = time.perf_counter() - t0
    errs, maxabs = [], 0.0
    for s, ref in zip(wl.segments, outs):
        got = y_gpu[s.offset:s.offset + s.rows * s.n].astype(np.float64).reshape(s.rows, s.n)
        nr = np.linalg.norm(ref, axis=1)
        ok = nr > 0
        errs.append(np.linalg.norm(got - ref, axis=1)[ok] / nr[ok])
        maxabs = max(maxabs, float(np.abs(got - ref).max()))
    e = np.concatenate(errs)
    return {"baseline": {"value": wl.total_samples / dt / 1e9, "unit": "GSamples/s",
                         "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                         "sample": "the whole workload (all 2^20 rows), one pass, plans excluded; "
                                   "FP64 numpy/BLAS on all host cores"},
            "err": {"normwise_rel_max": float(e.max()), "normwise_rel_mean": float(e.mean()),
                    "max_abs": maxabs, "snr_db_mean": float(np.mean(-20 * np.log10(np.maximum(e, 1e-300))))}}


def run_reference(args):
    """Reference arm: the FP64 oracle on the host, same workload, bounded steps."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import cauchy
    from synthetic import mixed_size_workload
    wl = mixed_size_workload()
    plans = {(n, u): cauchy.make_plan(n, v, rho) for n, ups in wl.updates.items()
             for u, (v, rho) in enumerate(ups)}

    def step():
        for s in wl.segments:
            xs = wl.x[s.offset:s.offset + s.rows * s.n].astype(np.float64).reshape(s.rows, s.n)
            cauchy.transform(plans[(s.n, s.update)], xs)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    value = wl.total_samples / dt / 1e9
    cores = len(os.sched_getaffinity(0))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GSamples/s",
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "rows": int(wl.total_rows), "samples": int(wl.total_samples),
                       "segments": len(wl.segments), "parallelism": "host cores (FP64 oracle)"},
            "cpu_baseline": {"value": value, "unit": "GSamples/s", "cores": cores, "kind": "oracle",
                             "sample": "the whole workload per step (FP64 Cauchy-formula oracle, "
                                       "numpy/BLAS on the host cores, plans excluded)"},
            "e2e": {"value": value, "unit": "GSamples/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-extra", action="store_true", help="skip the n=1024 and comparator items")
    ap.add_argument("--no-cpu", action="store_true",
                    help="skip the CPU oracle baseline and the oracle error checks of the extra lines")
    ap.add_argument("--quick", action="store_true", help="only the n=1024 large-n item")
    ap.add_argument("--only", choices=["n256", "n1024", "n4096", "n16384", "pruned", "backward", "fp64"],
                    help="run just this secondary line (for profiling one kernel family); prints "
                         "its JSON object alone")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.only:
        run_only(args)
    else:
        run_ours(args)


def run_only(args):
    """One secondary line without the headline step (profiling aid)."""
    import torch
    import paper_2409_08970_gb300 as pkg
    from paper_2409_08970_gb300 import build as _build
    _build.build()
    peaks = load_peaks()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream()
    flush_buf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def flush():
        flush_buf.fill_(1.0)

    D, H, G, R = pkg.CAUCHY_DENSE, pkg.CAUCHY_HIER, pkg.CAUCHY_DENSE_GFT, pkg.CAUCHY_NFST
    HL, HT = (H, 1), (H, 2)
    large = {"n256": (256, 4096, [HL, HT, D, G, R]), "n1024": (1024, 4096, [HL, HT, D, G, R]),
             "n4096": (4096, 4096, [HL, HT, D, G, R]), "n16384": (16384, 512, [HL, HT])}
    if args.only in large:
        n, batch, modes = large[args.only]
        out = bench_large(pkg, torch, dev, stream, args, flush, peaks, n, batch, modes, not args.no_cpu)
    elif args.only == "pruned":
        out = bench_pruned(pkg, torch, dev, stream, args, flush, peaks)
    elif args.only == "fp64":
        out = bench_fp64_n64(pkg, torch, dev, stream, args, flush, peaks)
    else:
        out = bench_backward(pkg, torch, dev, stream, args, flush, peaks)
    print(json.dumps({args.only: out}), flush=True)


if __name__ == "__main__":
    main()
