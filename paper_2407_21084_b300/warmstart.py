"""Learned warm start of the Picard iteration.

The paper has no counterpart: Algorithm 1 starts from ybar_N = g and sweeps
backwards; a Picard iteration starts from an initial iterate, y == 0 by
default. Here a small MLP (inputs: the wave vector s padded to 6, sigma0, a,
t_i; 3 x 256 GELU hidden units; output: the coefficient row alpha_i as
|Gamma| reals) is trained on coefficients the plain scheme itself produced
for random members of the d = 6 workload family, and its prediction replaces
y == 0. The iteration is unchanged, so a poor prediction costs iterations,
never accuracy. Network training and inference run in libqrmc's own kernels
(qr_mlp_*); this module only marshals arrays.

    python -m paper_2407_21084_b300.warmstart --train 2048 --heldout 256
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import time

import numpy as np

from . import _lib as L
from . import workloads as W

FP64, FP32 = L.QR_FP64, L.QR_FP32


# --------------------------------------------------------------- network
class MLP:
    """FP32 multilayer perceptron living in libqrmc (qr_mlp_*)."""

    def __init__(self, n_in, n_out, width=256, depth=3, max_batch=1024, seed=5, stream=None):
        """stream: a torch.cuda.Stream; default the current stream. The
        library's kernels and the binding's own tensor work (batch gathers,
        copies) both run on it, in order."""
        import torch

        self._L = L.load()
        self.n_in, self.n_out, self.max_batch = n_in, n_out, max_batch
        self.dims = [n_in] + [width] * depth + [n_out]
        self._ts = stream if stream is not None else torch.cuda.current_stream()
        self._h = C.c_void_p()
        st = self._L.qr_mlp_create(C.byref(self._h), n_in, width, depth, n_out, max_batch, seed,
                                   C.c_void_p(self._ts.cuda_stream))
        if st != L.QR_OK:
            msg = self._L.qr_mlp_last_error(self._h).decode() if self._h else ""
            self.close()
            raise L.QrError(st, msg)
        self.x_mu = np.zeros(n_in, dtype=np.float32)
        self.x_sd = np.ones(n_in, dtype=np.float32)
        self.y_mu = np.zeros(n_out, dtype=np.float32)
        self.y_sd = np.ones(n_out, dtype=np.float32)

    def _check(self, st):
        if st != L.QR_OK:
            raise L.QrError(st, self._L.qr_mlp_last_error(self._h).decode())

    @property
    def num_params(self) -> int:
        return int(self._L.qr_mlp_num_params(self._h))

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.num_params, dtype=np.float32)
        self._check(self._L.qr_mlp_get_params(self._h, p.ctypes.data_as(C.POINTER(C.c_float))))
        return p

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(self._L.qr_mlp_set_params(self._h, p.ctypes.data_as(C.POINTER(C.c_float))))

    @staticmethod
    def _dev(a):
        import torch

        return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda().contiguous()

    def gradients(self, X, T):
        """Gradient of mean((y - T)^2) on raw (unstandardised) arrays."""
        import torch

        with torch.cuda.stream(self._ts):
            return self._gradients(X, T)

    def _gradients(self, X, T):
        x, t = self._dev(X), self._dev(T)
        g = np.zeros(self.num_params, dtype=np.float32)
        loss = C.c_float()
        self._check(self._L.qr_mlp_gradients(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(t.data_ptr()),
                                             x.shape[0], g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(loss)))
        return g, float(loss.value)

    def forward_raw(self, X) -> np.ndarray:
        import torch

        with torch.cuda.stream(self._ts):
            return self._forward_raw(X)

    def _forward_raw(self, X) -> np.ndarray:
        import torch

        x = self._dev(X)
        y = torch.empty((x.shape[0], self.n_out), dtype=torch.float32, device="cuda")
        self._check(self._L.qr_mlp_forward(self._h, C.c_void_p(x.data_ptr()), x.shape[0], C.c_void_p(y.data_ptr())))
        return y.cpu().numpy()

    def fit(self, X, Y, steps=2000, batch=512, lr=1e-3, seed=0, lr_final=1e-5, target_scale="global"):
        """Adam on standardised inputs/outputs with a cosine learning rate. Returns the loss history.

        target_scale "global" divides every output by one common scale, so the
        loss weighs each coefficient by its own size (the large, low-frequency
        coefficients decide the sup error of the series; the small ones are
        mostly Monte Carlo noise of the training solves); "per_output"
        standardises each output on its own."""
        import torch

        with torch.cuda.stream(self._ts):
            return self._fit(X, Y, steps, batch, lr, seed, lr_final, target_scale)

    def _fit(self, X, Y, steps, batch, lr, seed, lr_final, target_scale):
        import torch

        X = np.asarray(X, dtype=np.float64)
        Y = np.asarray(Y, dtype=np.float64)
        self.x_mu, self.x_sd = X.mean(0).astype(np.float32), (X.std(0) + 1e-6).astype(np.float32)
        y_sd = Y.std(0) + 1e-6 if target_scale == "per_output" else np.full(Y.shape[1], (Y - Y.mean(0)).std() + 1e-6)
        self.y_mu, self.y_sd = Y.mean(0).astype(np.float32), y_sd.astype(np.float32)
        Xs = torch.as_tensor(((X - self.x_mu) / self.x_sd).astype(np.float32)).cuda()
        Ys = torch.as_tensor(((Y - self.y_mu) / self.y_sd).astype(np.float32)).cuda()
        rng = np.random.default_rng(seed)
        batch = min(batch, self.max_batch, X.shape[0])
        hist = []
        for it in range(steps):
            idx = torch.as_tensor(rng.choice(X.shape[0], size=batch, replace=False)).cuda()
            xb, yb = Xs[idx].contiguous(), Ys[idx].contiguous()
            cur = lr_final + 0.5 * (lr - lr_final) * (1 + np.cos(np.pi * it / max(1, steps)))
            loss = C.c_float()
            self._check(self._L.qr_mlp_train_step(self._h, C.c_void_p(xb.data_ptr()), C.c_void_p(yb.data_ptr()),
                                                  batch, float(cur), C.byref(loss) if it % 50 == 0 else None))
            if it % 50 == 0:
                hist.append(float(loss.value))
        return hist

    def predict(self, X) -> np.ndarray:
        X = np.asarray(X, dtype=np.float64)
        out = []
        for a in range(0, X.shape[0], self.max_batch):
            xs = ((X[a:a + self.max_batch] - self.x_mu) / self.x_sd).astype(np.float32)
            out.append(self.forward_raw(xs).astype(np.float64) * self.y_sd + self.y_mu)
        return np.concatenate(out)

    def close(self):
        if getattr(self, "_h", None):
            self._L.qr_mlp_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


# ------------------------------------------------------ coefficient rows
def alpha_to_rows(alpha: np.ndarray) -> np.ndarray:
    """(N, |Gamma|) complex -> (N, |Gamma|) reals: alpha_0, then (re, im) of the half set."""
    nG = alpha.shape[1]
    z = (nG - 1) // 2
    half = alpha[:, z + 1:]
    return np.concatenate([alpha[:, z:z + 1].real, np.stack([half.real, half.imag], -1).reshape(len(alpha), -1)], 1)


def rows_to_alpha(rows: np.ndarray) -> np.ndarray:
    nG = rows.shape[1]
    z = (nG - 1) // 2
    half = rows[:, 1:].reshape(len(rows), z, 2)
    a = np.zeros((len(rows), nG), dtype=np.complex128)
    a[:, z] = rows[:, 0]
    a[:, z + 1:] = half[..., 0] + 1j * half[..., 1]
    a[:, :z] = np.conj(a[:, z + 1:][:, ::-1])
    return a


# ----------------------------------------------------------- the family
def family_member(base: W.Workload, rng, M: int, seed: int) -> W.Workload:
    """s ~ U[-1,1]^d, sigma0 ~ U[0.2,0.6], a ~ U[0,0.5] around a base workload."""
    return base.with_(s=rng.uniform(-1.0, 1.0, size=base.d), sigma0=float(rng.uniform(0.2, 0.6)),
                      a=float(rng.uniform(0.0, 0.5)), M=M, seed=seed)


def features(w: W.Workload, width_s: int = 6) -> np.ndarray:
    """Rows (t_i, i = 0..N-1) of [s padded to width_s, sigma0, a, t_i]."""
    s = np.zeros(width_s)
    s[: w.d] = w.s
    t = np.arange(w.N) * w.T / w.N
    return np.column_stack([np.tile(s, (w.N, 1)), np.full(w.N, w.sigma0), np.full(w.N, w.a), t])


def solve(w: W.Workload, precision=FP32, stream=None) -> np.ndarray:
    from .solver import Solver

    with Solver.from_workload(w, precision=precision, stream=stream) as s:
        s.backward_sweep()
        return s.coefs()


def training_set(base: W.Workload, n: int, M: int, seed: int = 5):
    rng = np.random.default_rng(seed)
    X, Y = [], []
    for q in range(n):
        w = family_member(base, rng, M, seed=1000 + q)
        X.append(features(w))
        Y.append(alpha_to_rows(solve(w)))
    return np.concatenate(X), np.concatenate(Y)


def sup_error(s, pts, y_ref) -> float:
    """max over rows i and test points of |ybar_i(x) - y_ref_i(x)|."""
    return max(float(np.abs(s.eval(i, x) - y_ref[i]).max()) for i, x in enumerate(pts))


def iterate_to(s, pts, y_ref, tol, max_iter):
    """Picard iterations until the sup error against y_ref is <= tol.
    Returns (iterations, seconds spent in the iterations, final error)."""
    import torch

    t_iter = 0.0
    err = sup_error(s, pts, y_ref)
    q = 0
    while err > tol and q < max_iter:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.picard_step(1)
        t_iter += time.perf_counter() - t0
        q += 1
        err = sup_error(s, pts, y_ref)
    return q, t_iter, err


def study(base: W.Workload, n_train=2048, train_paths=2 ** 16, n_heldout=256, eval_paths=2 ** 18, n_fp64=16,
          steps=3000, tol=1e-3, test_points=1024, other_cloud=True, target_scale="global", log=None) -> dict:
    """Iterations and time to a sup error `tol` from y == 0 (FP64 and FP32
    forms) and from the network's start (FP32), on held-out members of the
    family of `base`.

    The reference of a problem is the fixed point of its own clouds (one
    backward sweep, Algorithm 1, equals N Picard iterations), in FP32; for
    the first n_fp64 problems the FP64 sweep is computed too and the FP64
    plain form is iterated, and the distance between the two references is
    reported. With other_cloud, the FP32 iteration also starts from the same
    problem's fixed point on an independent cloud (another seed): no start
    computed without the evaluation cloud can be closer to its fixed point
    than the cloud-independent solution, of which this start is an unbiased
    estimate, so its iteration count bounds what any warm start can save."""
    import torch

    from .solver import Solver

    t0 = time.perf_counter()
    X, Y = training_set(base, n_train, train_paths)
    t_data = time.perf_counter() - t0
    net = MLP(X.shape[1], Y.shape[1], max_batch=1024)
    t0 = time.perf_counter()
    hist = net.fit(X, Y, steps=steps, target_scale=target_scale)
    t_fit = time.perf_counter() - t0
    rng = np.random.default_rng(6)
    rows, ref_gap = [], 0.0
    for q in range(n_heldout):
        w = family_member(base, rng, eval_paths, seed=900000 + q)
        with Solver.from_workload(w, precision=FP32) as ref:
            ref.backward_sweep()
            pts = [ref.test_points(i, test_points) for i in range(w.N)]
            y_ref = [ref.eval(i, x) for i, x in enumerate(pts)]
        res = {}
        if q < n_fp64:
            with Solver.from_workload(w, precision=FP64) as r64:
                r64.backward_sweep()
                ref_gap = max(ref_gap, sup_error(r64, pts, y_ref))
        starts = [("fp32_cold", FP32, None), ("fp32_warm", FP32, "net")]
        if q < n_fp64:
            starts = [("fp64_cold", FP64, None)] + starts
        if other_cloud:
            starts.append(("fp32_other_cloud", FP32, "cloud"))
        for name, prec, start in starts:
            with Solver.from_workload(w, precision=prec) as s:
                if start == "net":
                    s.set_coefs(rows_to_alpha(net.predict(features(w))))
                elif start == "cloud":
                    with Solver.from_workload(w.with_(seed=w.seed + 7777777), precision=FP32) as o:
                        o.backward_sweep()
                        s.set_coefs(o.coefs())
                it, secs, err = iterate_to(s, pts, y_ref, tol, w.N + 2)
                res[name] = {"iterations": it, "seconds": secs, "sup_error": err}
        rows.append(res)
        if log and (q + 1) % 16 == 0:
            log("held-out %d/%d" % (q + 1, n_heldout))
    names = ["fp64_cold", "fp32_cold", "fp32_warm"] + (["fp32_other_cloud"] if other_cloud else [])
    summ = {}
    for k in names:
        sel = [r[k] for r in rows if k in r]
        if sel:
            its = np.array([x["iterations"] for x in sel])
            summ[k] = {"iterations_mean": float(its.mean()), "iterations_min": int(its.min()),
                       "iterations_max": int(its.max()),
                       "seconds_mean": float(np.mean([x["seconds"] for x in sel])), "problems": len(sel)}
    cold, warm = summ["fp32_cold"], summ["fp32_warm"]
    out = {"train_solves": n_train, "train_paths": train_paths, "target_scale": target_scale, "data_s": t_data,
           "fit_s": t_fit, "loss_first": hist[0], "loss_last": hist[-1], "heldout": n_heldout,
           "eval_paths": eval_paths, "tol": tol, "reference": "FP32 backward sweep of the same clouds",
           "fp64_vs_fp32_reference_sup": ref_gap if n_fp64 else None, "summary": summ,
           "iterations_saved_by_network": cold["iterations_mean"] - warm["iterations_mean"],
           "seconds_saved_by_network": cold["seconds_mean"] - warm["seconds_mean"]}
    if other_cloud:
        out["iterations_saved_by_other_cloud_fixed_point"] = \
            cold["iterations_mean"] - summ["fp32_other_cloud"]["iterations_mean"]
    if "fp64_cold" in summ:
        # the same problems in both forms: the first n_fp64
        w64 = [r for r in rows if "fp64_cold" in r]
        f64 = float(np.mean([r["fp64_cold"]["seconds"] for r in w64]))
        out["speedup_fp32_warm_vs_fp64_cold"] = f64 / max(1e-12, float(np.mean([r["fp32_warm"]["seconds"] for r in w64])))
        out["speedup_fp32_cold_vs_fp64_cold"] = f64 / max(1e-12, float(np.mean([r["fp32_cold"]["seconds"] for r in w64])))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2048, help="training solves")
    ap.add_argument("--train-paths", type=int, default=2 ** 16)
    ap.add_argument("--heldout", type=int, default=256)
    ap.add_argument("--heldout-fp64", type=int, default=16, help="held-out problems also solved in the FP64 form")
    ap.add_argument("--eval-paths", type=int, default=2 ** 18)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--tol", type=float, default=1e-3)
    ap.add_argument("--test-points", type=int, default=1024)
    ap.add_argument("--target-scale", choices=("global", "per_output"), default="global")
    ap.add_argument("--no-other-cloud", action="store_true")
    args = ap.parse_args()
    import sys

    out = study(W.c3(), args.train, args.train_paths, args.heldout, args.eval_paths, args.heldout_fp64, args.steps,
                args.tol, args.test_points, not args.no_other_cloud, args.target_scale,
                log=lambda m: print(m, file=sys.stderr, flush=True))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
