"""The fused FP64 CholeskyQR (one cooperative launch per orthonormalisation) that
the mixed-precision subspace iteration uses: on matrices whose condition number
spans 1 to 1e12 (the squared spectra a power step produces), at the shapes of the
D=8, chi=256 move and ragged ones, Q must have orthonormal columns to FP64 level
and span exactly the columns of Y (Q Q^T Y = Y); repeated calls give bitwise the
same Q (the Gram partials are reduced in a fixed order)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_08212_gb300 import ctm as C
    C.load()
    return C


def _matrix(rows, n, cond, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((rows, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = cond ** (-np.arange(n) / max(n - 1, 1))
    return (U * s) @ V.T * 3.7


@pytest.mark.parametrize("rows,n,cond,passes", [(2048, 256, 1e2, 3), (2048, 256, 1e8, 3),
                                                (2048, 256, 1e12, 4), (1000, 77, 1e6, 3),
                                                (16384, 256, 1e10, 3), (4000, 400, 1e4, 2),
                                                (33, 33, 10.0, 2), (512, 512, 1e3, 3)])
def test_fused_cholqr_orthonormal_and_same_span(ctm, rows, n, cond, passes):
    Y = _matrix(rows, n, cond, rows + n)
    rc, Q = ctm.ctm_cholqr_test(Y, passes)
    assert rc == ctm.OK
    orth = np.abs(Q.T @ Q - np.eye(n)).max()
    Yn = Y / np.linalg.norm(Y, axis=0)
    span = np.abs(Q @ (Q.T @ Yn) - Yn).max()
    print(f"cholqr {rows}x{n} cond {cond:.0e} passes {passes}: |Q^T Q - I| {orth:.1e}, "
          f"span residual {span:.1e}")
    assert orth < 1e-13
    # an ill-conditioned Y only determines its span to cond * eps
    assert span < max(1e-12, 1e-15 * cond)


def test_fused_cholqr_is_deterministic(ctm):
    Y = _matrix(2048, 256, 1e6, 3)
    rc1, Q1 = ctm.ctm_cholqr_test(Y, 3)
    rc2, Q2 = ctm.ctm_cholqr_test(Y, 3)
    assert rc1 == rc2 == ctm.OK
    assert np.array_equal(Q1, Q2)


def test_fused_cholqr_rank_deficient_columns_are_completed(ctm):
    """Three columns that repeat earlier ones: the unshifted passes flag them and
    replace them with random directions, so Q is still an orthonormal basis that
    contains span(Y)."""
    rng = np.random.default_rng(9)
    Y = rng.standard_normal((500, 40))
    Y[:, 10] = Y[:, 3]
    Y[:, 20] = 2 * Y[:, 5] - Y[:, 7]
    Y[:, 39] = Y[:, 0]
    rc, Q = ctm.ctm_cholqr_test(Y, 3)
    assert rc == ctm.OK
    assert np.abs(Q.T @ Q - np.eye(40)).max() < 1e-13
    assert np.abs(Q @ (Q.T @ Y) - Y).max() < 1e-10 * np.abs(Y).max()
