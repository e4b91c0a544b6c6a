"""The 5th-generation tensor-core building block of the shared-point group
kernel (tcgen05.mma, swizzled shared-memory operands, TMEM accumulator)
against the same product computed on the host from the same BF16 values."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def bf16_bits(x):
    """Round float32 values to BF16 (nearest even) and return the bit patterns."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    r = ((u >> 16) & 1) + 0x7FFF
    return ((u + r) >> 16).astype(np.uint16)


def bf16_val(b):
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("seed", [0, 1])
def test_tc_mma_tile_matches_host_product(seed):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_21084_b300 import _lib, build

    build.build()
    rng = np.random.default_rng(seed)
    A = bf16_bits(rng.normal(size=(128, 64)))
    B = bf16_bits(rng.normal(size=(32, 64)))
    D = _lib.tc_selftest(A, B)
    ref = bf16_val(A) @ bf16_val(B).T  # exact products, FP64 sums
    assert np.abs(D - ref).max() <= 1e-5 * np.abs(ref).max()
    # a layout mistake (a swapped chunk, a transposed operand) moves whole
    # products around; single-entry patterns pin every (row, k) position
    A1 = np.zeros((128, 64), dtype=np.uint16)
    B1 = np.zeros((32, 64), dtype=np.uint16)
    r, k = np.arange(128), (np.arange(128) * 7) % 64
    A1[r, k] = bf16_bits(np.ones(128) + r / 128.0)
    B1[np.arange(32), (np.arange(32) * 7) % 64] = bf16_bits(np.full(32, 2.0))
    D1 = _lib.tc_selftest(A1, B1)
    assert np.array_equal(D1, (bf16_val(A1) @ bf16_val(B1).T).astype(np.float32))
