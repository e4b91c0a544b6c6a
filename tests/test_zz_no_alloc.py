"""qr_project_static: the projection for callers that cannot allocate device
memory during the call (fixed memory budgets, latency-bound loops, code that
runs under another allocator). It keeps its partial sums in a fixed array
inside the library instead of context memory. Checked against the projection
that qr_picard_step runs on the same responses, on two calls in a row that
reuse the shared array, and against the FP64 oracle's iteration of the same
rows from the same previous iterate -- for a context on the table-driven
projection (d=2, |k|_inf<=4) and one on the compiled tiled projection (d=6,
|k|_1<=5).

This file is collected last on purpose: a run that stops at the first
failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

from paper_2407_21084_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-4}  # relative, normwise: FP64 plain form / FP32 precision form

CASES = {
    # workload, M, (lo, hi) of the two calls
    "c1_table": (W.c1, 3000, ((0, 8), (2, 5))),  # ragged M: not a multiple of the block or chunk size
    "c3_tree": (W.c3, 4500, ((29, 32), (30, 32))),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec", [0, 1])
def test_project_static_matches_picard_projection(prec, case, ora):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_21084_b300 import _lib, build, solver

    build.build()
    lib = _lib.load()
    mk, M, calls = CASES[case]
    w = mk()
    K = ora.gamma_list(w.gamma_kind, w.d, w.gamma_n)
    p = ora.Problem(d=w.d, N=w.N, T=w.T, k=K, b=w.b, sigma=w.sigma, f_kind=ora.F_CUBIC_MANUF, f_par=w.f_par,
                    g_kind=ora.GT_COS, g_par=w.g_par, M=M, seed=w.seed, clamp_L=w.clamp_L)
    with solver.Solver.from_workload(w, precision=prec, M=M) as s:
        s.picard_step(1)
        a_prev = s.coefs()
        s.picard_step(1)  # responses of the second iteration use a nonzero iterate
        ref = s.coefs()
        lo_all = min(lo for lo, _ in calls)
        hi_all = max(hi for _, hi in calls)
        a_ora, _ = ora.picard_iter(p, a_prev, i_range=(lo_all, hi_all))
        rows = np.stack([s.responses(i) if lo_all <= i < hi_all else np.zeros(M) for i in range(w.N)])
        dt = torch.float32 if prec == 1 else torch.float64
        S_dev = torch.from_numpy(rows).to(dtype=dt, device="cuda").contiguous()
        for lo, hi in calls:  # two calls in a row on the shared scratch
            out = torch.full((hi - lo, s.nG, 2), float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            st = lib.qr_project_static(s._ctx, C.c_void_p(S_dev[lo:hi].data_ptr()), lo, hi,
                                       C.c_void_p(out.data_ptr()))
            assert st == 0, lib.qr_last_error(s._ctx)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            got = got[..., 0] + 1j * got[..., 1]
            err = np.abs(got - ref[lo:hi]).max() / np.abs(ref[lo:hi]).max()
            assert err < TOL[prec], err
            err_ora = np.abs(got - a_ora[lo:hi]).max() / np.abs(a_ora[lo:hi]).max()
            assert err_ora < TOL[prec], err_ora
        # sizes beyond the fixed scratch are refused with a message
        big = solver.Solver.from_workload(w.with_(N=200), precision=prec, M=2 ** 18)
        try:
            st = lib.qr_project_static(big._ctx, C.c_void_p(S_dev.data_ptr()), 0, 200,
                                       C.c_void_p(out.data_ptr()))
            assert st == 1
            assert b"scratch" in lib.qr_last_error(big._ctx)
        finally:
            big.close()
