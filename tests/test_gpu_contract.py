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
