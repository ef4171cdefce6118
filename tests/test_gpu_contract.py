"""The contraction kernels against numpy: the FP64 leg-map GEMM and the tcgen05
TF32 / BF16 GEMM (FP32 accumulation), on ragged shapes that span several tiles
and the K, M and N tails."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [(128, 64, 64), (200, 130, 70), (256, 256, 512), (1000, 300, 1000), (129, 257, 9),
          (4096, 64, 128), (384, 2048, 256)]
# Frobenius-relative error bars: FP64 round-off; TF32 (10-bit mantissa) and
# BF16 (7-bit mantissa) operand rounding with FP32 accumulation on N(0,1) data
TOL = {0: 1e-13, 1: 2e-3, 2: 1e-2}


@pytest.fixture(scope="module")
def ctm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_08212_gb300 import ctm as C
    C.load()
    return C


def _bf16(x):
    """float64 -> nearest bfloat16 (ties to even), as float64: the operand packing's
    one rounding, written from the format (1 + 7 significand bits kept)."""
    b = np.asarray(x, dtype=np.float64).view(np.uint64)
    sign = b & np.uint64(1 << 63)
    mag = b & np.uint64((1 << 63) - 1)
    low = mag & np.uint64((1 << 45) - 1)
    keep = mag >> np.uint64(45)
    half = np.uint64(1 << 44)
    up = (low > half) | ((low == half) & ((keep & np.uint64(1)) == np.uint64(1)))
    return (((keep + up.astype(np.uint64)) << np.uint64(45)) | sign).view(np.float64)


def _tf32(x):
    """float64 -> float32 (nearest, ties to even) -> TF32 (10 fraction bits, ties
    away from zero), as float64: the operand packing of the TF32 mode."""
    u = np.asarray(x, dtype=np.float64).astype(np.float32).view(np.uint32)
    sign = u & np.uint32(0x80000000)
    mag = ((u & np.uint32(0x7FFFFFFF)) + np.uint32(0x1000)) & np.uint32(0xFFFFE000)
    return (mag | sign).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("shape", SHAPES)
def test_contract_elementwise(ctm, precision, shape):
    """Element by element against the product of the rounded operands computed in
    FP64: what is left is the accumulation error, bounded per element by
    K 2^-18 sum_k |a_ik b_kj| for FP32 accumulation (32 times the worst case of
    truncating additions) or K 2^-50 sum_k |a_ik b_kj| for FP64, plus one unit in
    the last place of a rounded operand for a tie the packing may break the other
    way."""
    M, N, K = shape
    rng = np.random.default_rng(M * 11 + N * 5 + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    rc, C = ctm.ctm_contract_test(precision, A, B)
    assert rc == ctm.OK
    rnd = {0: lambda x: x, 1: _tf32, 2: _bf16}[precision]
    Ar, Br = rnd(A), rnd(B)
    ref = Ar @ Br
    absprod = np.abs(Ar) @ np.abs(Br)
    if precision == 0:
        bound = K * 2.0 ** -50 * absprod + 1e-300
    else:
        ulp = {1: 2.0 ** -10, 2: 2.0 ** -7}[precision]
        bound = K * 2.0 ** -18 * absprod + ulp * (np.abs(Ar).max(axis=1)[:, None] *
                                                  np.abs(Br).max(axis=0)[None, :])
    err = np.abs(C - ref)
    worst = np.unravel_index(np.argmax(err / bound), err.shape)
    assert np.all(err <= bound), (worst, err[worst], bound[worst])


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("shape", SHAPES)
def test_contract_against_numpy(ctm, precision, shape):
    M, N, K = shape
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    rc, C = ctm.ctm_contract_test(precision, A, B)
    assert rc == ctm.OK
    ref = A @ B
    err = np.linalg.norm(C - ref) / np.linalg.norm(ref)
    assert err < TOL[precision], err
    if precision != 0:
        # the error is operand rounding, not a layout fault: it is far below 1
        # and every row and column is populated
        assert np.all(np.abs(C).sum(axis=1) > 0) and np.all(np.abs(C).sum(axis=0) > 0)
