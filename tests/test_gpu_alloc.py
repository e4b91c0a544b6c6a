"""Device memory of a context through the caller's allocator (qr_opts
dev_alloc / dev_free): from Python the binding passes PyTorch's caching
allocator, so the context's buffers show up in torch's accounting while it
lives and go back when it is destroyed; the iteration is the same bit for bit
as with the library's own stream-ordered allocation."""
import numpy as np
import pytest

from paper_2407_21084_b300 import workloads as W

pytestmark = pytest.mark.gpu


def test_context_memory_through_torch_allocator():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_21084_b300 import build, solver

    build.build()
    w = W.c2()
    M = 2 ** 16
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    s = solver.Solver.from_workload(w, precision=1, M=M)
    inside = torch.cuda.memory_allocated()
    # at least the responses (N x M floats) and the partial sums live in torch's pool
    assert inside - before >= w.N * M * 4
    s.picard_step(2)
    a = s.coefs()
    s.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before
    with solver.Solver(w.d, w.N, w.T, w.nu_kind, w.mu, w.gamma_kind, w.gamma_n, w.b, w.sigma,
                       solver.L.QR_F_CUBIC_MANUF, w.f_par, solver.L.QR_GT_COS, w.g_par, M, w.seed, precision=1,
                       clamp_L=w.clamp_L, torch_memory=False) as own:
        assert torch.cuda.memory_allocated() == before
        own.picard_step(2)
        assert np.array_equal(own.coefs().view(np.float64), a.view(np.float64))
