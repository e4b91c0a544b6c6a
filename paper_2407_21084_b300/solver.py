"""Python face of libqrmc: one Solver per QRMC problem.

PyTorch is used only for device memory (device-pointer evaluation) and for
the CUDA stream the library launches on; all arithmetic runs in libqrmc.
"""
from __future__ import annotations

import ctypes as C
import json
import time

import numpy as np

from . import _lib as L
from .workloads import Sec5Problem, Workload


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Solver:
    """A QRMC problem on the GPU (wraps a qr_ctx)."""

    def __init__(self, d, N, T, nu_kind, mu, gamma_kind, gamma_n, b, sigma, f_kind, f_par, g_kind, g_par, M,
                 seed, precision=L.QR_FP64, clamp_L=0.0, stream=None, lattice_n=0, instance=0, path_kernel=0,
                 damping_q=0.0, torch_memory=True):
        self._L = L.load()
        self.shard_world = 1
        self.d, self.N, self.T, self.M = int(d), int(N), float(T), int(M)
        self.precision = precision
        b = np.ascontiguousarray(b, dtype=np.float64)
        sigma = np.ascontiguousarray(sigma, dtype=np.float64).reshape(-1)
        if b.size != d or sigma.size != d * d:
            raise ValueError("b needs d and sigma d*d entries (d = %d)" % d)
        fp = np.ascontiguousarray(np.atleast_1d(f_par), dtype=np.float64)
        gp = np.ascontiguousarray(np.atleast_1d(g_par), dtype=np.float64)
        self._keep = (b, sigma, fp, gp)
        # the problem as constructed (a checkpoint stores it beside the coefficients)
        self._config = dict(d=int(d), N=int(N), T=float(T), nu_kind=int(nu_kind), mu=float(mu),
                            gamma_kind=int(gamma_kind), gamma_n=int(gamma_n), b=b.tolist(), sigma=sigma.tolist(),
                            f_kind=int(f_kind), f_par=fp.tolist(), g_kind=int(g_kind), g_par=gp.tolist(), M=int(M),
                            seed=int(seed), precision=int(precision), clamp_L=float(clamp_L),
                            lattice_n=int(lattice_n), instance=int(instance), path_kernel=int(path_kernel),
                            damping_q=float(damping_q))
        self.iterations_done = 0  # Picard iterations (or sweeps) behind the current coefficients
        nu = L.QrNu(nu_kind, mu)
        gam = L.QrGamma(gamma_kind, gamma_n)
        f = L.QrFn(f_kind, _dp(fp), fp.size)
        g = L.QrFn(g_kind, _dp(gp), gp.size)
        if stream is None:
            stream_ptr = None
            try:
                import torch

                if torch.cuda.is_available():
                    stream_ptr = torch.cuda.current_stream().cuda_stream
            except Exception:  # noqa: BLE001 - torch is optional plumbing
                stream_ptr = None
        else:
            stream_ptr = stream
        self.damping_q = float(damping_q)
        # device buffers from PyTorch's caching allocator (the library's own
        # stream-ordered allocation when torch_memory is False)
        alloc, free = L.torch_allocator() if torch_memory and stream_ptr is not None else (None, None)
        opts = L.QrOpts(M, seed, precision, clamp_L, stream_ptr,
                        L.QR_U_LATTICE if lattice_n else L.QR_U_PHILOX, lattice_n, instance, path_kernel,
                        self.damping_q, alloc, free, None)
        self._ctx = C.c_void_p()
        st = self._L.qr_init(C.byref(self._ctx), d, N, T, C.byref(nu), C.byref(gam), _dp(b), _dp(sigma),
                             C.byref(f), C.byref(g), C.byref(opts))
        if st != L.QR_OK:
            msg = self._L.qr_last_error(self._ctx).decode() if self._ctx else ""
            self.close()
            raise L.QrError(st, msg)
        n = C.c_int()
        L.check(self._L.qr_gamma_size(self._ctx, C.byref(n)), self._ctx)
        self.nG = n.value

    @classmethod
    def from_workload(cls, w: Workload, precision=L.QR_FP64, M=None, stream=None, clamp=True, path_kernel=0,
                      instance=0):
        return cls(w.d, w.N, w.T, w.nu_kind, w.mu, w.gamma_kind, w.gamma_n, w.b, w.sigma, L.QR_F_CUBIC_MANUF,
                   w.f_par, L.QR_GT_COS, w.g_par, w.M if M is None else M, w.seed, precision=precision,
                   clamp_L=w.clamp_L if clamp else 0.0, stream=stream, path_kernel=path_kernel, instance=instance)

    @classmethod
    def from_sec5(cls, p: Sec5Problem, precision=L.QR_FP64, M=None, stream=None, instance=0, path_kernel=0):
        """The test problem of Sec. 5 (Student or Cauchy nu, min/sin driver and
        terminal condition, cosine basis, damping exponent p.q), no truncation."""
        return cls(p.d, p.N, p.T, p.nu_kind, p.mu, p.gamma_kind, p.gamma_n, p.b, p.sigma,
                   L.QR_F_PAPER_MIN, p.f_par, L.QR_GT_PAPER_SIN, p.g_par, p.M if M is None else M, p.seed,
                   precision=precision, clamp_L=0.0, stream=stream, instance=instance, path_kernel=path_kernel,
                   damping_q=p.q)

    def cosine_coefs(self):
        """For a context of the cosine basis (N^d set): the multi-indices of
        Gamma (canonical order) and the real cosine coefficients a_k of every row."""
        return self.gamma_list(), self.coefs().real

    # -------------------------------------------------------------- calls
    def picard_step(self, n_iter: int = 1) -> float:
        r = C.c_double()
        L.check(self._L.qr_picard_step(self._ctx, n_iter, C.byref(r)), self._ctx)
        self.iterations_done += n_iter
        return r.value

    def backward_sweep(self):
        L.check(self._L.qr_backward_sweep(self._ctx), self._ctx)
        self.iterations_done += self.N

    def evals_per_iteration(self) -> int:
        """path.coef evaluations of one Picard iteration: M |Gamma| N(N+1)/2."""
        return self.M * self.nG * self.N * (self.N + 1) // 2

    def iterate(self, n_iter: int, log=None, tol: float | None = None) -> list:
        """Picard iterations one at a time with a metrics record each: wall
        seconds (the step waits for its device work), path.coef evaluations
        per second, the residual max |alpha^(q) - alpha^(q-1)|, and the clamp
        hits and non-finite responses of that iteration. Records are appended
        to `log` (a path or a text file object) as JSON lines. Stops early
        once the residual is <= tol."""
        out = []
        fh = open(log, "a") if isinstance(log, str) else log
        try:
            for _ in range(n_iter):
                before = self.stats()
                t0 = time.perf_counter()
                r = self.picard_step(1)
                sec = time.perf_counter() - t0
                after = self.stats()
                rec = {"iteration": self.iterations_done, "seconds": sec,
                       "path_coef_evals_per_s": self.evals_per_iteration() / sec, "residual": r,
                       "clamp_hits": after["clamp_hits"] - before["clamp_hits"],
                       "nonfinite": after["nonfinite"] - before["nonfinite"]}
                out.append(rec)
                if fh is not None:
                    fh.write(json.dumps(rec) + "\n")
                    fh.flush()
                if tol is not None and r <= tol:
                    break
        finally:
            if isinstance(log, str):
                fh.close()
        return out

    # ------------------------------------------------------- checkpoints
    def save_checkpoint(self, path: str):
        """The Picard state (the FP64 coefficient rows, the iterations behind
        them and the problem as constructed) to an .npz file. The iteration is
        a function of the previous coefficients and of counter-based random
        numbers that do not depend on the iteration, so a solver resumed from
        the file continues bit-identically."""
        np.savez(path, coefs=self.coefs(), iterations=np.int64(self.iterations_done),
                 config=np.array(json.dumps(self._config)))

    @classmethod
    def load_checkpoint(cls, path: str, stream=None) -> "Solver":
        z = np.load(path)
        cfg = json.loads(str(z["config"]))
        cfg["b"] = np.asarray(cfg["b"])
        cfg["sigma"] = np.asarray(cfg["sigma"])
        s = cls(**cfg, stream=stream)
        s.set_coefs(z["coefs"])
        s.iterations_done = int(z["iterations"])
        return s

    def inject_fault(self, kind: int):
        """Arm one host-side fault (L.QR_FAULT_ALLOC, _LAUNCH, _NAN; see qr_inject_fault)."""
        L.check(self._L.qr_inject_fault(self._ctx, int(kind)), self._ctx)

    def coefs(self) -> np.ndarray:
        a = np.zeros((self.N, self.nG), dtype=np.complex128)
        L.check(self._L.qr_get_coefs(self._ctx, _dp(a.view(np.float64))), self._ctx)
        return a

    def set_coefs(self, alpha: np.ndarray):
        a = np.ascontiguousarray(alpha, dtype=np.complex128)
        assert a.shape == (self.N, self.nG)
        L.check(self._L.qr_set_coefs(self._ctx, _dp(a.view(np.float64))), self._ctx)

    def gamma_list(self) -> np.ndarray:
        k = np.zeros((self.nG, self.d), dtype=np.int32)
        L.check(self._L.qr_gamma_list(self._ctx, k.ctypes.data_as(C.POINTER(C.c_int))), self._ctx)
        return k

    def responses(self, i: int) -> np.ndarray:
        S = np.zeros(self.M)
        L.check(self._L.qr_get_responses(self._ctx, i, _dp(S)), self._ctx)
        return S

    def eval(self, i: int, x):
        """ybar_i at the rows of x: numpy (host path) or a CUDA torch tensor (device path)."""
        try:
            import torch
        except ImportError:  # pragma: no cover
            torch = None
        if torch is not None and isinstance(x, torch.Tensor) and x.is_cuda:
            xs = x.contiguous().to(torch.float64)
            y = torch.empty(xs.shape[0], dtype=torch.float64, device=xs.device)
            L.check(self._L.qr_eval(self._ctx, i, C.c_void_p(xs.data_ptr()), xs.shape[0],
                                    C.c_void_p(y.data_ptr()), L.QR_DEVICE), self._ctx)
            return y
        xs = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
        y = np.zeros(xs.shape[0])
        L.check(self._L.qr_eval(self._ctx, i, C.c_void_p(xs.ctypes.data), xs.shape[0], C.c_void_p(y.ctypes.data),
                                L.QR_HOST), self._ctx)
        return y

    def test_points(self, i: int, n: int) -> np.ndarray:
        """n nu-distributed test points of time index i (Philox test tag), shape (n, d)."""
        x = np.zeros((n, self.d))
        L.check(self._L.qr_test_points(self._ctx, i, n, _dp(x)), self._ctx)
        return x

    def mse_indicators(self, exact, n: int = 1000) -> dict:
        """MSE_max and MSE_av of Sec. 5, eq. (mse): natural logs of the mean
        squared error of ybar_i against exact(t_i, x) at n test points per i
        (with damping, of the damped ybar^q_i against exact / (1 + |x|^2)^{q/2})."""
        per_i = []
        for i in range(self.N):
            x = self.test_points(i, n)
            ex = exact(i * self.T / self.N, x)
            if self.damping_q:
                ex = ex / (1.0 + (x * x).sum(axis=1)) ** (self.damping_q / 2)
            e = self.eval(i, x) - ex
            per_i.append(float(np.mean(e * e)))
        per_i = np.array(per_i)
        return {"mse_max": float(np.log(per_i.max())), "mse_av": float(np.log(per_i.mean())), "points": n}

    # ------------------------------------------- one problem over several GPUs
    def shard(self, rank: int, world: int):
        """Restrict this context to its rank's path chunks (qr_shard)."""
        L.check(self._L.qr_shard(self._ctx, rank, world), self._ctx)
        self.shard_world = world

    def shard_groups(self):
        """(group sums as a CUDA float64 tensor (8, N, |Gamma_+|, 2) aliasing the
        library's array, g_lo, g_hi): this rank fills groups [g_lo, g_hi)."""
        import torch

        ptr, nb = C.c_void_p(), C.c_longlong()
        gl, gh = C.c_int(), C.c_int()
        L.check(self._L.qr_shard_groups(self._ctx, C.byref(ptr), C.byref(nb), C.byref(gl), C.byref(gh)), self._ctx)
        if not ptr.value:
            raise L.QrError(L.QR_EINVAL, "the context is not sharded")
        ngp = nb.value // (16 * self.N)
        view = _DeviceArray(ptr.value, (8, self.N, ngp, 2), "<f8")
        return torch.as_tensor(view, device="cuda"), gl.value, gh.value

    def picard_begin(self):
        L.check(self._L.qr_picard_begin(self._ctx), self._ctx)

    def picard_finish(self) -> float:
        r = C.c_double()
        L.check(self._L.qr_picard_finish(self._ctx, C.byref(r)), self._ctx)
        return r.value

    def picard_step_sharded(self, group=None) -> float:
        """One Picard iteration of a problem sharded over the ranks of a
        torch.distributed process group: own paths and group sums, the
        all-gather of the group sums, then the common reduction."""
        import torch

        self.picard_begin()
        buf, gl, gh = self.shard_groups()
        torch.cuda.synchronize()  # this rank's group sums are on the context's stream
        exchange_group_sums(buf, gl, gh, self.shard_world, group)
        torch.cuda.synchronize()
        return self.picard_finish()

    def set_profiling(self, on: bool = True):
        L.check(self._L.qr_set_profiling(self._ctx, 1 if on else 0), self._ctx)

    def stats(self) -> dict:
        s = L.QrStats()
        L.check(self._L.qr_get_stats(self._ctx, C.byref(s)), self._ctx)
        return {f: getattr(s, f) for f, _ in L.QrStats._fields_}

    def close(self):
        if getattr(self, "_ctx", None):
            self._L.qr_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class _DeviceArray:
    """A device pointer with its shape, seen by torch through __cuda_array_interface__."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def exchange_group_sums(buf, g_lo: int, g_hi: int, world: int, group=None):
    """All-gather of the group sums of a sharded iteration: buf is the
    (8, ...) array of group sums with this rank's groups [g_lo, g_hi) filled;
    afterwards every group is filled, rank r's groups at [r 8/W, (r+1) 8/W).
    Works on CUDA tensors (NCCL) and CPU tensors (gloo) alike."""
    import torch
    import torch.distributed as dist

    per = 8 // world
    mine = buf[g_lo:g_hi].contiguous()
    parts = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    for r, t in enumerate(parts):
        buf[r * per:(r + 1) * per].copy_(t)


def tree_layout(kind: int, d: int, n: int):
    """The slot map of the compile-time tree kernels (host only, no device):
    idx (slots, 2, T) int and coef (slots, 2, T) float, see qr_tree_layout."""
    lib = L.load()
    ns, nt = C.c_int(), C.c_int()
    L.check(lib.qr_tree_layout(kind, d, n, C.byref(ns), C.byref(nt), None, None))
    idx = np.zeros((ns.value, 2, nt.value), dtype=np.int32)
    coef = np.zeros((ns.value, 2, nt.value))
    L.check(lib.qr_tree_layout(kind, d, n, C.byref(ns), C.byref(nt), idx.ctypes.data_as(C.POINTER(C.c_int)),
                               _dp(coef)))
    return idx, coef


def philox_words(ctr_key: np.ndarray) -> np.ndarray:
    """Device Philox4x32-10 on rows (ctr0..3, key0, key1) -> rows of 4 words."""
    lib = L.load()
    a = np.ascontiguousarray(ctr_key, dtype=np.uint32).reshape(-1, 6)
    out = np.zeros((a.shape[0], 4), dtype=np.uint32)
    L.check(lib.qr_philox_words(a.ctypes.data_as(C.POINTER(C.c_uint32)), a.shape[0],
                                out.ctypes.data_as(C.POINTER(C.c_uint32))))
    return out


def sample_normals_tree(d, seed, instance, i, m0, n, j):
    """FP32 normals of the tree path kernels, shape (n, d)."""
    lib = L.load()
    z = np.zeros((n, d))
    L.check(lib.qr_sample_normals_tree(d, seed, instance, i, m0, n, j, _dp(z)))
    return z


def sample(d, nu_kind, mu, seed, instance, i, m0, n, j, precision=L.QR_FP64):
    """Device sampler: (u, x, z) arrays of shape (n, d)."""
    lib = L.load()
    u = np.zeros((n, d))
    x = np.zeros((n, d))
    z = np.zeros((n, d))
    nu = L.QrNu(nu_kind, mu)
    L.check(lib.qr_sample(d, C.byref(nu), seed, instance, i, m0, n, j, precision, _dp(u), _dp(x), _dp(z)))
    return u, x, z
