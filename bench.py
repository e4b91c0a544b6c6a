"""Benchmark of one QRMC Picard iteration (arXiv 2407.21084) on B300.

A step is one Jacobi-Picard iteration of the whole hot path on the d=6
precision-form workload (N=32 time steps, M=2^22 paths per time step,
Gamma = {|k|_1 <= 5} of Z^6 with 3653 coefficients, FP32 path and basis
arithmetic, FP64 cross-block sums): path-and-series kernel, projection,
deterministic reduction. The metric is path.coef evaluations per second,
M |Gamma| N(N+1)/2 per iteration; seconds per iteration are reported too.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves an independent instance of the same
workload (distinct Philox instance field); there is no data-path collective,
only a barrier and a max over ranks for the timing ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2407_21084_b300 import workloads as W  # noqa: E402

PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")


def cpu_model() -> str:
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def measure_peaks(dev: int, stream) -> dict:
    """FMA throughput of this device's FP32 and FP64 pipes, measured in
    process by the library's FMA-chain kernels (qr_fma_peak): a burst of
    about 60 ms and a run of about 2 s per kind, with the SM clocks sampled
    meanwhile. The FP32 peak is the larger of the scalar and the packed
    two-lane form and of the two interleaved."""
    from paper_2407_21084_b300 import _lib as L

    out = {}
    with ClockSampler(dev) as clk:
        for name, kind in (("fp32", L.QR_PEAK_FP32), ("fp32x2", L.QR_PEAK_FP32X2),
                           ("fp32mix", L.QR_PEAK_FP32MIX), ("fp64", L.QR_PEAK_FP64)):
            b = L.fma_peak(kind, 60.0, stream.cuda_stream)
            su = L.fma_peak(kind, 2000.0, stream.cuda_stream)
            out[name] = {"burst_tflops": b["tflops"], "sustained_tflops": su["tflops"], "sustained_ms": su["ms"]}
            out["sm_count"] = su["sm_count"]
    out["clocks"] = clk.summary()
    out["how"] = ("qr_fma_peak: resident 256-thread CTAs on every SM, 8 independent FMA chains per thread, "
                  "~20 ms launches timed with CUDA events: ~60 ms (burst) and ~2 s (sustained) per kind")
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev: int):
        self.dev = dev
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms: float, ws: int) -> float:
    """Job time of a replica run: the slowest rank's time (all-reduce MAX;
    on the GPU tensor for NCCL, on a CPU tensor for gloo)."""
    if ws == 1:
        return ms
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(evals_per_step: float, ms_step: float, ws: int) -> float:
    """Whole-job throughput of ws replicas, each doing evals_per_step per step."""
    return ws * evals_per_step / (ms_step / 1e3)


def cpu_baseline(w: W.Workload, alpha_prev: np.ndarray, rows, m_sample: int, gpu_rows: dict | None):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample:
    rows `rows` of one Picard iteration from alpha_prev over the first
    m_sample paths. Returns (baseline dict, reference alpha rows)."""
    import oracle

    oracle.build()
    K = oracle.gamma_list(w.gamma_kind, w.d, w.gamma_n)
    p = oracle.Problem(d=w.d, N=w.N, T=w.T, k=K, b=w.b, sigma=w.sigma, f_kind=oracle.F_CUBIC_MANUF,
                       f_par=w.f_par, g_kind=oracle.GT_COS, g_par=w.g_par, M=m_sample, seed=w.seed,
                       clamp_L=w.clamp_L)
    evals = 0.0
    ref = {}
    t0 = time.perf_counter()
    for i in rows:
        a, _ = oracle.picard_iter(p, alpha_prev, i_range=(i, i + 1), m_range=(0, m_sample))
        ref[i] = a[i]
        evals += m_sample * len(K) * (w.N - i)  # series at N-1-i points + one projection
    dt = time.perf_counter() - t0
    cores = min(oracle.max_threads(), -(-m_sample // 1024))  # one chunk of >= 1024 paths per thread
    base = {"value": evals / dt, "unit": "path.coef evals/s", "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(), "host_threads": os.cpu_count(),
            "sample": "rows i=%s of one Picard iteration, first %d of %d paths, FP64 oracle (OpenMP), %.1f s"
                      % (list(rows), m_sample, w.M, dt)}
    return base, ref, p


def bench_c4(stream, steps: int, flush) -> dict:
    """The many-instance workload: 256 problems of uneven d, |Gamma| and N
    (M = 2^18 each, 64 of them sharing their sample points) advanced by one
    batched Picard iteration per step (persistent path kernel, tensor-core
    shared-point kernel, projections). Device time with CUDA events on the
    batch's stream (L2 flushed before each step; the batch's state, ~10 GB,
    is far larger than L2 anyway), and end to end through the C-ABI with
    every instance's coefficients copied from and back to host memory."""
    import torch

    from paper_2407_21084_b300 import batch as B

    ws_ = W.c4()
    t0 = time.perf_counter()
    sol = B.solvers_for(ws_, stream.cuda_stream)
    b = B.Batch(sol)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    b.picard_step(1)  # autotuning of tiles and grid, then the first iteration
    t_tune = time.perf_counter() - t0
    b.picard_step(1)
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.picard_step(1)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    evals = sum(w.evals_per_iter() for w in ws_)
    host = [s.coefs() for s in sol]
    io = sum(a.nbytes for a in host)
    e2e = []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s, a in zip(sol, host):
            s.set_coefs(a)
        b.picard_step(1)
        host = [s.coefs() for s in sol]
        e2e.append(time.perf_counter() - t0)
    info = b.info()
    b.close()
    for s in sol:
        s.close()
    ms_step = float(np.mean(ms))
    return {"workload": "c4_256_instances_M262144", "instances": len(ws_),
            "shared_point_instances": info["grouped_instances"], "shared_groups": info["shared_groups"],
            "dims": sorted(set(w.d for w in ws_)),
            "n_gamma_range": [min(w.n_gamma() for w in ws_), max(w.n_gamma() for w in ws_)],
            "evals_per_iteration": evals, "s_per_batch_iteration": ms_step / 1e3,
            "path_coef_evals_per_s": evals / (ms_step / 1e3), "steps": steps,
            "autotune": {"tiles_per_item": info["tiles_per_item"], "grid": info["grid"], "s": t_tune},
            "setup_s": t_setup,
            "e2e": {"value": evals / float(np.mean(e2e)), "unit": "path.coef evals/s",
                    "h2d_bytes_per_step": io, "d2h_bytes_per_step": io}}


def bench_warm_start() -> dict:
    """The learned warm start and the precision form, bounded to under a
    minute: a network trained on 96 plain FP32 solves of the d=6 family
    (2^14 paths each), then 3 held-out problems (2^16 paths) iterated to a
    1e-3 sup error against the fixed point of their own clouds, from y == 0
    in the FP64 plain form and in the FP32 form, and from the network's start
    in the FP32 form; wall time of the iterations (device work and the
    per-iteration accuracy check). The full study (2048 training solves, 256
    held-out problems) is python -m paper_2407_21084_b300.warmstart."""
    from paper_2407_21084_b300 import warmstart as WS

    t0 = time.perf_counter()
    out = WS.study(W.c3(), n_train=96, train_paths=2 ** 14, n_heldout=3, eval_paths=2 ** 16, n_fp64=3, steps=600,
                   tol=1e-3, test_points=512, other_cloud=True)
    out["wall_s"] = time.perf_counter() - t0
    return out


def run_reference(args, w):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    N = w.N
    alpha0 = np.zeros((N, W.gamma_size(w.gamma_kind, w.d, w.gamma_n)), dtype=complex)
    rows = [N - 1, N // 2, N // 4]
    times, vals = [], []
    base = None
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        base, _, _ = cpu_baseline(w, alpha0, rows, args.ref_paths, None)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            vals.append(base["value"])
    v = float(np.median(vals))
    line = {"impl": "reference", "metric": "path_coef_evals_per_s", "value": v, "unit": "path.coef evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "d": w.d, "N": w.N, "M": w.M, "n_gamma": w.n_gamma(),
                       "sample": base["sample"]},
            "cpu_baseline": base,
            "e2e": {"value": v, "unit": "path.coef evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(W.CONFIGS))
    ap.add_argument("--ref-paths", type=int, default=98304, help="paths of the oracle sample (10-25 s on 8-16 cores)")
    ap.add_argument("--paths", type=int, default=0, help="override M (profiling captures only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-c4", action="store_true", help="skip the many-instance (config 4) key")
    ap.add_argument("--no-warm", action="store_true", help="skip the warm-start / precision-form key")
    args = ap.parse_args()
    w = W.CONFIGS[args.workload]()
    if args.paths:
        w = w.with_(M=args.paths)

    if args.impl == "reference":
        return run_reference(args, w)

    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_2407_21084_b300 import solver

    prec = solver.L.QR_FP32
    dev = torch.cuda.current_device()
    # a dedicated stream: the library launches on it (one CUDA graph per
    # iteration) and the timing events are recorded on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s = solver.Solver(w.d, w.N, w.T, w.nu_kind, w.mu, w.gamma_kind, w.gamma_n, w.b, w.sigma,
                      solver.L.QR_F_CUBIC_MANUF, w.f_par, solver.L.QR_GT_COS, w.g_par, w.M, w.seed,
                      precision=prec, clamp_L=w.clamp_L, instance=rank, stream=stream.cuda_stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (126 MB)
    peaks = measure_peaks(dev, stream)

    for _ in range(args.warmup):
        s.picard_step(1)
    torch.cuda.synchronize()
    # per-kernel times: the library's events on its stream, over timed-size
    # steps run with profiling on (direct launches); the step time itself is
    # taken below on the graph-launched iteration
    s.set_profiling(True)
    st0 = s.stats()
    for _ in range(args.steps):
        flush.zero_()
        s.picard_step(1)
    st1 = s.stats()
    s.set_profiling(False)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = []
    alpha_prev = None
    with ClockSampler(dev) as clk:
        for k in range(args.steps):
            flush.zero_()
            if k == args.steps - 1:
                alpha_prev = s.coefs()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.picard_step(1)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
    total_ms = max_over_ranks(float(np.sum(step_ms)), ws)
    if ws > 1:
        dist.barrier()
    evals = w.evals_per_iter()
    ms_step = total_ms / args.steps
    value = job_value(evals, ms_step, ws)

    # dominant kernel: the path-and-series kernel, timed by the library's
    # events on its launch stream over the timed region
    n_paths = st1["launches_paths"] - st0["launches_paths"]
    ms_paths = (st1["ms_paths"] - st0["ms_paths"]) / max(1, n_paths)
    ms_proj = (st1["ms_project"] - st0["ms_project"]) / max(1, n_paths)
    ms_red = (st1["ms_reduce"] - st0["ms_reduce"]) / max(1, n_paths)
    nG = w.n_gamma()
    pairs = (nG + 1) / 2.0
    series_points = w.M * w.N * (w.N - 1) / 2.0
    flops_paths = series_points * pairs * 8.0  # 4 FP32 FMA per pair (complex Horner step)
    clocks = clk.summary()
    # roofline denominator: the FP32 FMA rate measured on this device, the
    # sustained figure (the path kernel runs ~0.8 s launches back to back
    # inside a long timed region), the larger of scalar and packed FMA
    pk = peaks
    fp32_forms = ("fp32", "fp32x2", "fp32mix")
    peak = max(pk[f]["sustained_tflops"] for f in fp32_forms)
    peak_burst = max(pk[f]["burst_tflops"] for f in fp32_forms)
    achieved = flops_paths / (ms_paths / 1e3) / 1e12
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic_paths_c3.json")
    if os.path.exists(tfile):
        try:
            tj = json.load(open(tfile))
            if tj.get("kernel_source_hash") == _kernel_hash():
                traffic = tj["bytes_per_full_launch"]
        except (OSError, ValueError, KeyError):
            traffic = None

    # end to end through the C-ABI with host buffers: H2D of the previous
    # iterate, the iteration, D2H of the new coefficients, every step
    e2e_ms = []
    a_host = s.coefs()
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.set_coefs(a_host)
        s.picard_step(1)
        a_host = s.coefs()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_val = job_value(evals, max_over_ranks(float(np.mean(e2e_ms)), ws), ws)
    io_bytes = w.N * nG * 16

    line = {
        "metric": "path_coef_evals_per_s", "value": value, "unit": "path.coef evals/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "s_per_picard_iteration": ms_step / 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "d": w.d, "N": w.N, "M": w.M, "n_gamma": nG, "gamma": "|k|_1<=5",
                   "precision": "fp32 path/basis, fp64 cross-block sums and alpha",
                   "l2": "flushed (256 MB write) between timed steps", "parallelism": "replicas" if ws > 1 else "1gpu"},
        "kernels_ms": {"paths": ms_paths, "project": ms_proj, "reduce": ms_red},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "k_paths_tree (path-and-series)",
                     "peak_basis": "measured FP32 FMA rate of this device, sustained (~2 s of FMA chains, "
                                   "qr_fma_peak), max of scalar, packed two-lane and interleaved FMA; of measured",
                     "peak_burst": peak_burst, "frac_of_burst": achieved / peak_burst,
                     "work": "M N(N-1)/2 series points x (|Gamma|+1)/2 pairs x 8 flop"},
        "fp32_peak_measured": {"sustained_tflops": peak, "burst_tflops": peak_burst,
                               "scalar": pk["fp32"], "packed_x2": pk["fp32x2"], "mixed": pk["fp32mix"]},
        "fp64_peak_measured": pk["fp64"],
        "sm_count": pk["sm_count"],
        "peak_clocks": pk["clocks"],
        "clocks": clocks,
        "gpu_launches": 4 * args.steps,  # per iteration: path, projection, reduction, tree repack
        "e2e": {"value": e2e_val, "unit": "path.coef evals/s", "h2d_bytes_per_step": io_bytes,
                "d2h_bytes_per_step": io_bytes},
    }
    # accuracy against the exact solution of the manufactured PDE: the
    # indicators of Sec. 5, eq. (mse), at 1000 test points per time index
    line["mse_vs_exact"] = s.mse_indicators(lambda t, x: w.exact_u(t, x), n=1000)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rows = [w.N - 1, w.N // 2, w.N // 4]
        base, ref, p = cpu_baseline(w, alpha_prev, rows, args.ref_paths, None)
        line["cpu_baseline"] = base
        # sup error of the FP32 GPU form against the FP64 oracle on the same
        # sample (same previous iterate, same first paths)
        g = solver.Solver(w.d, w.N, w.T, w.nu_kind, w.mu, w.gamma_kind, w.gamma_n, w.b, w.sigma,
                          solver.L.QR_F_CUBIC_MANUF, w.f_par, solver.L.QR_GT_COS, w.g_par, args.ref_paths, w.seed,
                          precision=prec, clamp_L=w.clamp_L)
        g.set_coefs(alpha_prev)
        g.picard_step(1)
        ag = g.coefs()
        import oracle

        sup = 0.0
        for i in rows:
            x = oracle.test_points(p, i, w.n_test)
            sup = max(sup, float(np.abs(g.eval(i, x) - oracle.series(p, ref[i], x)).max()))
        g.close()
        line["sup_error_vs_fp64_oracle"] = {"value": sup, "test_points": w.n_test, "rows": rows,
                                            "paths": args.ref_paths}
    if rank == 0 and ws == 1 and not args.no_c4:
        line["c4_batch"] = bench_c4(stream, max(2, min(args.steps, 5)), flush)
    if rank == 0 and ws == 1 and not args.no_warm:
        line["warm_start"] = bench_warm_start()
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def _kernel_hash() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in ("qr_fast.cu", "qr_fast.h", "qr_tree.cuh", "qr_device.cuh", "qr_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_2407_21084_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    sys.exit(main())
