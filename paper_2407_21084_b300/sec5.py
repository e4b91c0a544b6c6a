"""The paper's own experiments of Sec. 5 on this implementation.

Test problem: dX = dW, g = 1 + kappa + sin(lam sum x), f = min(1, [y - kappa
- 1 - sin(lam sum x) e^{lam^2 d (t-T)/2}]^2), kappa = 0.6, lam = 1/sqrt(d),
T = 1, Student nu (mu = 2), cosine basis on Gamma_F (d = 1), Gamma_T or
Gamma_H, damping exponents q of eq. (yqi), one backward sweep (Algorithm 1) in FP32 as in
the paper. For each timed row of the paper's FP32 tables (d = 1, 2, 3, 5, 7,
9, 11; the rows the paper timed above `--max-gpu-s` seconds, among them
d = 9 and 11, only when that limit is raised), prints one JSON line with

* the wall time of one backward sweep here (CUDA-synchronised) and the
  paper's GPU time with the hardware it names (one GTX TITAN Black, Kepler,
  FP32, CUDA 7.5; four of them for the d = 5 and 7 rows), and W = M |Gamma| N(N+1)/2 path.coef evaluations per
  second for both;
* MSE_max and MSE_av of eq. (mse) against the exact solution (1000 test
  points per time index; damped by (1 + |x|^2)^{q/2} for q > 0), averaged
  over `--runs` independent runs, for each damping exponent q the paper
  tabulates, beside the paper's values (averages over 10^3 runs);
* for the d = 1 rows with a printed interval: the 99 % confidence interval
  of ybar_0(0) over 50 runs beside the paper's (u(0,0) = 1.6).

    python -m paper_2407_21084_b300.sec5 [--rows d1,d2] [--runs 3]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import _lib as L
from . import workloads as W

# (label, d, kind, DEG or K, |Gamma|, Delta, M, paper GPU s, paper (MSE_max, MSE_av) by damping q, paper 99 % CI)
ROWS = [
    ("d1 K=100", 1, W.G_FULL_N, 100, 101, 0.05, 2 * 10 ** 4, 0.09,
     {0.0: (-3.658, -3.868), 2.1: (-4.615, -4.874), 5.1: (-4.517, -5.130), 8.1: (-4.781, -5.319)}, (1.578, 1.667)),
    ("d1 K=150", 1, W.G_FULL_N, 150, 151, 0.02, 2 * 10 ** 5, 7.37,
     {0.0: (-4.427, -4.900), 2.1: (-6.450, -6.740), 5.1: (-6.685, -7.094), 8.1: (-6.740, -7.221)}, (1.595, 1.624)),
    ("d1 K=200", 1, W.G_FULL_N, 200, 201, 0.01, 2 * 10 ** 6, 414.44,
     {0.0: (-4.704, -5.524), 2.1: (-8.465, -8.729), 5.1: (-8.717, -9.096), 8.1: (-8.830, -9.301)}, None),
    ("d2 Tot DEG20", 2, W.G_TOTAL_N, 20, 231, 0.05, 2 * 10 ** 4, 0.33, {0.0: (-2.322, -2.773), 5.1: (-4.646, -5.239)}, None),
    ("d2 Tot DEG25", 2, W.G_TOTAL_N, 25, 351, 0.02, 2 * 10 ** 5, 35.51, {0.0: (-2.869, -3.688), 5.1: (-6.761, -7.186)}, None),
    ("d2 Tot DEG31", 2, W.G_TOTAL_N, 31, 528, 0.01, 2 * 10 ** 6, 2243.06, {0.0: (-2.978, -3.966), 5.1: (-8.793, -9.107)}, None),
    ("d2 Hyp DEG19", 2, W.G_HYP_N, 19, 99, 0.05, 2 * 10 ** 4, 0.16, {0.0: (-2.526, -3.062), 5.1: (-5.588, -6.196)}, None),
    ("d2 Hyp DEG24", 2, W.G_HYP_N, 24, 133, 0.02, 2 * 10 ** 5, 12.38, {0.0: (-2.745, -3.550), 5.1: (-7.487, -8.191)}, None),
    ("d2 Hyp DEG30", 2, W.G_HYP_N, 30, 172, 0.01, 2 * 10 ** 6, 662.54, {0.0: (-2.898, -3.770), 5.1: (-9.389, -10.137)}, None),
    ("d3 Tot DEG22", 3, W.G_TOTAL_N, 22, 2300, 0.05, 2 * 10 ** 5, 53.89, {0.0: (-2.164, -2.785), 5.1: (-5.699, -6.141)}, None),
    ("d3 Hyp DEG20", 3, W.G_HYP_N, 20, 411, 0.05, 2 * 10 ** 5, 8.37, {0.0: (-2.255, -3.191), 5.1: (-6.883, -7.662)}, None),
    ("d3 Hyp DEG22", 3, W.G_HYP_N, 22, 459, 0.02, 2 * 10 ** 6, 592.19, {0.0: (-2.249, -3.356), 5.1: (-7.778, -8.875)}, None),
    # the d = 5 and d = 7 tables give the times of the paper's multi-GPU code (4 GPUs)
    ("d5 Tot DEG20", 5, W.G_TOTAL_N, 20, 53130, 0.2, 2 * 10 ** 6, 874.36,
     {0.0: (-1.906, -2.049), 5.1: (-6.537, -6.994)}, None, 4),
    ("d5 Tot DEG21", 5, W.G_TOTAL_N, 21, 65780, 0.1, 2 * 10 ** 7, 19163.72,
     {0.0: (-2.221, -3.356), 5.1: (-8.482, -9.103)}, None, 4),
    ("d5 Hyp DEG16", 5, W.G_HYP_N, 16, 3042, 0.2, 2 * 10 ** 6, 49.27,
     {0.0: (-2.353, -3.259), 5.1: (-7.312, -7.835)}, None, 4),
    ("d5 Hyp DEG17", 5, W.G_HYP_N, 17, 3122, 0.1, 2 * 10 ** 7, 773.70,
     {0.0: (-1.955, -3.278), 5.1: (-7.438, -8.125)}, None, 4),
    ("d5 Hyp DEG36", 5, W.G_HYP_N, 36, 10503, 0.1, 2 * 10 ** 7, 2718.07,
     {0.0: (-2.216, -3.494), 5.1: (-8.609, -9.407)}, None, 4),
    ("d5 Hyp DEG66", 5, W.G_HYP_N, 66, 24893, 0.1, 2 * 10 ** 7, 6563.77,
     {0.0: (-2.381, -3.603), 5.1: (-8.819, -9.703)}, None, 4),
    ("d7 Hyp DEG36", 7, W.G_HYP_N, 36, 94460, 0.1, 2 * 10 ** 7, 33284.41, {5.1: (-8.879, -9.574)}, None, 4),
    ("d9 Hyp DEG12", 9, W.G_HYP_N, 12, 102656, 0.1, 2 * 10 ** 7, 44437.40, {5.1: (-8.101, -8.359)}, None, 4),
    ("d11 Hyp DEG5", 11, W.G_HYP_N, 5, 75264, 0.1, 2 * 10 ** 8, 373816.97, {5.1: (-7.828, -8.785)}, None, 4),
]


def _problem(d, kind, n, delta, M, seed, q=0.0):
    return W.Sec5Problem(d=d, N=int(round(1.0 / delta)), gamma_kind=kind, gamma_n=n, M=M, seed=seed, q=q)


def run_row(row, runs: int, ci_runs: int, precision=L.QR_FP32, path_kernel=0, paths=None, profile=False):
    import torch

    from .solver import Solver

    label, d, kind, n, ng, delta, M, gpu_s, paper_mse, ci = row[:10]
    if paths:
        M = paths
    paper_gpus = row[10] if len(row) > 10 else 1
    times, mse, split = [], {}, []
    for q in paper_mse:
        per = []
        for r in range(runs):
            p = _problem(d, kind, n, delta, M, seed=1 + r, q=q)
            with Solver.from_sec5(p, precision=precision, path_kernel=path_kernel) as s:
                k, _ = s.cosine_coefs()
                assert len(k) == ng, (label, len(k), ng)
                if profile:
                    s.set_profiling(True)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                s.backward_sweep()
                torch.cuda.synchronize()
                if q == min(paper_mse):
                    times.append(time.perf_counter() - t0)
                    if profile:
                        st = s.stats()
                        split.append({k: st[k] for k in ("ms_paths", "ms_project", "ms_reduce")})
                per.append(s.mse_indicators(lambda t, x: p.exact_u(t, x), n=1000))
        mse[str(q)] = {"mse_max": float(np.mean([m["mse_max"] for m in per])),
                       "mse_av": float(np.mean([m["mse_av"] for m in per])),
                       "paper_mse_max": paper_mse[q][0], "paper_mse_av": paper_mse[q][1]}
    N = int(round(1.0 / delta))
    work = float(M) * ng * N * (N + 1) / 2.0
    t = float(np.median(times))
    out = {"row": label, "d": d, "gamma": {W.G_FULL_N: "Gamma_F", W.G_TOTAL_N: "Gamma_T", W.G_HYP_N: "Gamma_H"}[kind],
           "deg": n, "n_gamma": ng, "N": N, "M": M, "precision": "fp32" if precision == L.QR_FP32 else "fp64",
           "s_per_sweep": t, "evals_per_s": work / t,
           "paper_gpu_s": gpu_s, "paper_gpu_evals_per_s": work / gpu_s, "speedup_vs_paper_gpu": gpu_s / t,
           "paper_hardware": "%dx GeForce GTX TITAN Black (Kepler GK110), FP32, CUDA 7.5" % paper_gpus,
           "path_kernel": path_kernel, "mse_by_q": mse, "runs": runs}
    if paths:
        out["speedup_vs_paper_gpu"] = None
        out["note"] = "M overridden: the time is not comparable with the paper's"
    if profile:
        # per-kernel device time of the timed sweeps (events on the library's
        # stream, one synchronisation per kernel: the sweep is then slower)
        out["kernel_ms"] = split
    if ci is not None and ci_runs > 0:
        vals = []
        for r in range(ci_runs):
            p = _problem(d, kind, n, delta, M, seed=1001 + r)
            with Solver.from_sec5(p, precision=precision, path_kernel=path_kernel) as s:
                s.backward_sweep()
                vals.append(float(s.eval(0, np.zeros((1, d)))[0]))
        v = np.array(vals)
        half = 2.576 * v.std(ddof=1) / np.sqrt(len(v))
        out["ci99_y0"] = [float(v.mean() - half), float(v.mean() + half)]
        out["paper_ci99_y0"] = list(ci)
        out["ci_runs"] = ci_runs
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rows", default="d1,d2,d3,d5,d7,d9,d11", help="comma-separated prefixes of the row labels")
    ap.add_argument("--runs", type=int, default=3, help="independent runs per row for time and MSE")
    ap.add_argument("--ci-runs", type=int, default=50, help="runs for the d = 1 confidence intervals")
    ap.add_argument("--max-gpu-s", type=float, default=3000.0, help="skip rows the paper timed above this")
    ap.add_argument("--paths", type=int, default=0, help="override M of every row (0: the paper's M)")
    ap.add_argument("--profile", action="store_true", help="record per-kernel device times of the timed sweeps")
    ap.add_argument("--path-kernel", type=int, default=0,
                    help="0: automatic; 1: the unfolded set on the Fourier kernels; 2: the direct cosine kernels")
    args = ap.parse_args()
    want = [w.strip() for w in args.rows.split(",") if w.strip()]
    for row in ROWS:
        # a prefix ends at a non-digit: "d1" selects the d = 1 rows, not d = 11
        picked = any(row[0].startswith(w) and not row[0][len(w):len(w) + 1].isdigit() for w in want)
        if not picked or row[7] > args.max_gpu_s:
            continue
        try:
            out = run_row(row, args.runs, args.ci_runs, path_kernel=args.path_kernel, paths=args.paths or None,
                          profile=args.profile)
        except L.QrError as e:  # e.g. an unfolded set too large for the generic kernels' shared memory
            out = {"row": row[0], "skipped": str(e)}
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
