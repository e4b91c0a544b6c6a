"""The bounds-checked build (libqrmc_checked.so, QR_CHECKED=1): the hot
kernels test every computed index into the responses, the projection
partials and the coefficient rows against its buffer and report one that
falls outside as QR_ECUDA. Each route runs in it (table and tree kernels,
FP64 and FP32, the direct cosine kernels, the many-instance engine with its
tensor-core group) without a report, and gives the same coefficients bit
for bit as the normal build (the checks skip nothing)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_SCRIPT = r"""
import sys
sys.path.insert(0, {root!r})
import numpy as np
import torch
from paper_2407_21084_b300 import _lib, build
_lib.load({lib!r})
from paper_2407_21084_b300 import batch as B, solver, workloads as W

out = {{}}
with solver.Solver.from_workload(W.c1().with_(M=3000), precision=0) as s:
    s.picard_step(2)
    out["c1_fp64"] = s.coefs()
with solver.Solver.from_workload(W.c3().with_(M=5000, N=6), precision=1) as s:
    s.picard_step(2)
    out["c3_tree_fp32"] = s.coefs()
with solver.Solver.from_workload(W.c2().with_(M=4096), precision=1) as s:
    s.backward_sweep()
    out["c2_sweep_fp32"] = s.coefs()
for prec in (0, 1):
    p = W.Sec5Problem(d=5, N=3, gamma_kind=W.G_HYP_N, gamma_n=8, M=700, seed=2, q=5.1)
    with solver.Solver.from_sec5(p, precision=prec, path_kernel=2) as s:
        s.picard_step(1)
        out["cos_direct_%d" % prec] = s.coefs()
st = torch.cuda.Stream()
ws = W.c4(n_instances=10, n_shared=3, M=3000)
sol = B.solvers_for(ws, st.cuda_stream)
b = B.Batch(sol)
b.picard_step(1)
for q, s in enumerate(sol):
    out["batch_%d" % q] = s.coefs()
b.close()
for s in sol:
    s.close()
np.savez({dst!r}, **out)
print("ok")
"""


@pytest.fixture(scope="module")
def libs():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_21084_b300 import build

    build.build()
    build.build(checked=True)
    return build.LIB, build.LIB_CHECKED


def _run(lib, dst):
    r = subprocess.run([sys.executable, "-c", _SCRIPT.format(root=ROOT, lib=lib, dst=dst)], capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stderr[-3000:]
    return np.load(dst)


def test_checked_build_reports_nothing_and_matches(libs, tmp_path):
    plain = _run(libs[0], str(tmp_path / "plain.npz"))
    checked = _run(libs[1], str(tmp_path / "checked.npz"))
    assert sorted(plain.files) == sorted(checked.files)
    for k in plain.files:
        assert np.array_equal(plain[k].view(np.float64), checked[k].view(np.float64)), k
