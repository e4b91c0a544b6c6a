"""GPU tests of the learned warm start (no counterpart in the paper): the
network's gradients against the FP64 oracle network, training, and the gain
of the warm start over y == 0 on held-out problems."""
import numpy as np
import pytest

from paper_2407_21084_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ws():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_21084_b300 import build, warmstart

    build.build()
    return warmstart


def test_gradients_match_fp64_oracle(ws):
    from oracle import mlp as omlp

    rng = np.random.default_rng(0)
    net = ws.MLP(9, 37, width=48, depth=3, max_batch=64, seed=3)
    # random (not the initial) parameters, exactly representable in FP32
    p = (rng.normal(size=net.num_params) * 0.3).astype(np.float32)
    net.set_params(p)
    X = rng.normal(size=(29, 9)).astype(np.float32)  # ragged batch vs the 64x64 GEMM tiles
    T = rng.normal(size=(29, 37)).astype(np.float32)
    g, loss = net.gradients(X, T)
    lo, go = omlp.loss_and_grad(p.astype(np.float64), net.dims, X, T)
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    assert np.abs(g - go).max() <= 2e-5 * np.abs(go).max()
    y = net.forward_raw(X)
    yo = omlp.forward(p.astype(np.float64), net.dims, X)
    assert np.abs(y - yo).max() <= 1e-5 * np.abs(yo).max()


def test_training_fits_a_smooth_map(ws):
    rng = np.random.default_rng(1)
    X = rng.uniform(-1, 1, size=(2048, 4))
    Y = np.column_stack([np.sin(X @ rng.normal(size=4)), np.cos(2 * X[:, 0]) * X[:, 1], X[:, 2] ** 2])
    net = ws.MLP(4, 3, width=64, depth=3, max_batch=256, seed=2)
    hist = net.fit(X, Y, steps=1500, batch=256, lr=3e-3, target_scale="per_output")
    assert hist[-1] < 0.02 * hist[0]
    err = np.abs(net.predict(X[:200]) - Y[:200]).max()
    assert err < 0.1


def test_training_on_a_side_stream_equals_the_default_stream(ws):
    """The network runs on the torch stream current at its creation; trained
    there (a non-blocking stream whose batch gathers the library's kernels
    must wait for) it reaches exactly the parameters of the same training on
    the default stream."""
    import torch

    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, size=(1024, 5))
    Y = np.column_stack([np.sin(X @ rng.normal(size=5)), X[:, 0] * X[:, 1]])
    params = []
    for side in (False, True):
        st = torch.cuda.Stream() if side else torch.cuda.default_stream()
        with torch.cuda.stream(st):
            net = ws.MLP(5, 2, width=64, depth=3, max_batch=256, seed=6)
            net.fit(X, Y, steps=300, batch=256, lr=3e-3)
            params.append(net.get_params())
            assert np.isfinite(net.predict(X[:64])).all()
            net.close()
    assert np.array_equal(params[0], params[1])


def test_rows_round_trip(ws):
    rng = np.random.default_rng(2)
    K = np.array([[a, b] for a in range(-2, 3) for b in range(-2, 3)])
    half = rng.normal(size=(3, 12)) + 1j * rng.normal(size=(3, 12))
    a = np.zeros((3, 25), dtype=complex)
    a[:, 12] = rng.normal(size=3)
    a[:, 13:] = half
    a[:, :12] = np.conj(half[:, ::-1])
    assert np.allclose(ws.rows_to_alpha(ws.alpha_to_rows(a)), a)
    assert K.shape[0] == 25


def test_warm_start_needs_fewer_iterations(ws):
    """A d=2 family (|k|_inf<=4, N=8): a network trained on 48 plain solves
    starts held-out problems closer to their fixed point than y == 0."""
    from paper_2407_21084_b300.solver import Solver

    base = W.c1()
    X, Y = ws.training_set(base, 48, 2 ** 12, seed=11)
    net = ws.MLP(X.shape[1], Y.shape[1], width=128, depth=3, max_batch=256, seed=4)
    net.fit(X, Y, steps=1500, batch=256, lr=2e-3)
    rng = np.random.default_rng(12)
    cold_it, warm_it = [], []
    for q in range(4):
        w = ws.family_member(base, rng, 2 ** 14, seed=5000 + q)
        with Solver.from_workload(w, precision=0) as ref:
            ref.backward_sweep()
            pts = [ref.test_points(i, 256) for i in range(w.N)]
            y_ref = [ref.eval(i, x) for i, x in enumerate(pts)]
        for warm, out in ((False, cold_it), (True, warm_it)):
            with Solver.from_workload(w, precision=0) as s:
                if warm:
                    s.set_coefs(ws.rows_to_alpha(net.predict(ws.features(w))))
                it, _, err = ws.iterate_to(s, pts, y_ref, 1e-3, w.N + 2)
                assert err <= 1e-3
                out.append(it)
    assert np.mean(warm_it) < np.mean(cold_it)
