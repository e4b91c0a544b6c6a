"""Failure paths, checkpoint/resume and the per-iteration metrics log, on the
GPU without faulting it: every fault is armed on the host (qr_inject_fault or
the QR_FAULT environment variable) and taken by the library's own error
paths; afterwards the context must iterate exactly like a fresh one."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2407_21084_b300 import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mods():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_21084_b300 import _lib, build, solver

    build.build()
    return solver, _lib


def _bits(a):
    return np.ascontiguousarray(a).view(np.float64)


@pytest.mark.parametrize("prec", [0, 1])
def test_launch_fault_leaves_the_context_usable(mods, prec):
    solver, L = mods
    w = W.c1().with_(M=3000)
    with solver.Solver.from_workload(w, precision=prec) as s, solver.Solver.from_workload(w, precision=prec) as ref:
        s.inject_fault(L.QR_FAULT_LAUNCH)
        with pytest.raises(L.QrError) as e:
            s.picard_step(1)
        assert e.value.status == L.QR_ECUDA
        assert s.stats()["iterations"] == 0  # nothing ran
        s.picard_step(2)
        ref.picard_step(2)
        assert np.array_equal(_bits(s.coefs()), _bits(ref.coefs()))


@pytest.mark.parametrize("w", [W.c1().with_(M=2048), W.c3().with_(M=4096, N=6)], ids=["table", "tree"])
def test_nan_fault_is_reported_and_recovered_from_a_checkpoint(mods, w):
    solver, L = mods
    with solver.Solver.from_workload(w, precision=1) as s, solver.Solver.from_workload(w, precision=1) as ref:
        s.picard_step(1)
        saved = s.coefs()
        s.inject_fault(L.QR_FAULT_NAN)
        with pytest.raises(L.QrError) as e:
            s.picard_step(1)
        assert e.value.status == L.QR_ENONFINITE
        assert s.stats()["nonfinite"] > 0
        s.set_coefs(saved)
        s.picard_step(1)
        ref.picard_step(2)
        assert np.array_equal(_bits(s.coefs()), _bits(ref.coefs()))


def test_alloc_fault_fails_one_call(mods):
    solver, L = mods
    with solver.Solver.from_workload(W.c1().with_(M=1024), precision=0) as s:
        s.picard_step(1)
        x = np.zeros((5, 2))
        s.inject_fault(L.QR_FAULT_ALLOC)
        with pytest.raises(L.QrError) as e:
            s.eval(1, x)
        assert e.value.status == L.QR_ENOMEM
        y = s.eval(1, x)
        assert np.isfinite(y).all()


def test_unknown_fault_kind_is_rejected(mods):
    solver, L = mods
    with solver.Solver.from_workload(W.c1().with_(M=256), precision=0) as s:
        with pytest.raises(L.QrError) as e:
            s.inject_fault(9)
        assert e.value.status == L.QR_EINVAL


_ENV_SCRIPT = r"""
import sys
sys.path.insert(0, {root!r})
from paper_2407_21084_b300 import _lib as L, solver, workloads as W
try:
    s = solver.Solver.from_workload(W.c1().with_(M=512), precision=0)
except L.QrError as e:
    print("init", e.status)
    sys.exit(0)
print("init", 0)
try:
    s.picard_step(1)
    print("step", 0)
except L.QrError as e:
    print("step", e.status)
import numpy as np
s.set_coefs(np.zeros((s.N, s.nG), dtype=complex))  # the restart state (y == 0)
s.picard_step(1)
print("again", 0)
s.close()
"""


@pytest.mark.parametrize("fault,expect", [("alloc", ["init 2"]), ("launch", ["init 0", "step 3", "again 0"]),
                                          ("nan", ["init 0", "step 5", "again 0"])])
def test_fault_from_the_environment(mods, fault, expect):
    env = dict(os.environ, QR_FAULT=fault)
    r = subprocess.run([sys.executable, "-c", _ENV_SCRIPT.format(root=ROOT)], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.split("\n")[: len(expect)] == expect, r.stdout


@pytest.mark.parametrize("prec", [0, 1])
def test_checkpoint_resume_is_bit_identical(mods, tmp_path, prec):
    """One iteration, a checkpoint, a new context from the file and two more
    iterations give the coefficients of three uninterrupted iterations."""
    solver, L = mods
    w = W.c2().with_(M=5000)
    path = str(tmp_path / "state.npz")
    with solver.Solver.from_workload(w, precision=prec) as s:
        s.picard_step(1)
        s.save_checkpoint(path)
    with solver.Solver.load_checkpoint(path) as r:
        assert r.iterations_done == 1
        r.picard_step(2)
        resumed = r.coefs()
    with solver.Solver.from_workload(w, precision=prec) as ref:
        ref.picard_step(3)
        assert np.array_equal(_bits(resumed), _bits(ref.coefs()))


def test_iteration_log(mods, tmp_path):
    solver, L = mods
    w = W.c1().with_(M=4096)
    path = str(tmp_path / "progress.jsonl")
    with solver.Solver.from_workload(w, precision=1) as s:
        recs = s.iterate(6, log=path)
        coefs = s.coefs()
    lines = [json.loads(x) for x in open(path)]
    assert lines == recs and len(lines) == 6
    assert [r["iteration"] for r in lines] == list(range(1, 7))
    for r in lines:
        assert r["seconds"] > 0 and r["path_coef_evals_per_s"] > 0 and r["nonfinite"] == 0
    # Picard contracts on this problem: the residual falls over the iterations
    assert lines[-1]["residual"] < lines[0]["residual"]
    assert np.isfinite(coefs).all()
