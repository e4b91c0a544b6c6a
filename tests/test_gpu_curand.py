"""External known-answer check of the device Philox4x32-10 against cuRAND's
own Philox4_32_10 device generator on the same GPU: after curand_init(seed,
subsequence, offset) the first four words are Philox4x32-10 at counter
(offset/4 as 64 bits, subsequence as 64 bits) with key (seed lo, seed hi);
the library's generator must give the same words bit for bit."""
import ctypes as C
import os
import subprocess
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_lib():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = tempfile.mkdtemp(prefix="curand_ref_")
    so = os.path.join(d, "libcurandref.so")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-Xcompiler", "-fPIC",
                           "-shared", "-o", so, os.path.join(HERE, "curand_philox_ref.cu")])
    lib = C.CDLL(so)
    lib.curand_first4.restype = C.c_int
    lib.curand_first4.argtypes = [C.POINTER(C.c_ulonglong), C.c_int, C.POINTER(C.c_uint)]
    return lib


def test_philox_matches_curand(curand_lib):
    from paper_2407_21084_b300 import build, solver

    build.build()
    rng = np.random.default_rng(2024)
    n = 4096
    seed = rng.integers(0, 2 ** 63, size=n, dtype=np.uint64)
    sub = rng.integers(0, 2 ** 63, size=n, dtype=np.uint64)
    off = rng.integers(0, 2 ** 40, size=n, dtype=np.uint64) * np.uint64(4)
    rows = np.ascontiguousarray(np.stack([seed, sub, off], 1).astype(np.uint64))
    ref = np.zeros((n, 4), dtype=np.uint32)
    assert curand_lib.curand_first4(rows.ctypes.data_as(C.POINTER(C.c_ulonglong)), n,
                                    ref.ctypes.data_as(C.POINTER(C.c_uint))) == 0
    ctr = off // np.uint64(4)
    ck = np.stack([ctr & np.uint64(0xffffffff), ctr >> np.uint64(32), sub & np.uint64(0xffffffff),
                   sub >> np.uint64(32), seed & np.uint64(0xffffffff), seed >> np.uint64(32)], 1).astype(np.uint32)
    got = solver.philox_words(ck)
    assert np.array_equal(got, ref)
