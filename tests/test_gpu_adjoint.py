"""GPU adjoint of the truncated left singular vectors (ctm_svd_left_adjoint)
against the gradient oracle's (oracle.ctm_grad.svd_left_adjoint, itself pinned by
central differences and PyTorch's SVD backward): tall, wide and square matrices,
ragged sizes, the projector shapes of the D=8, chi=256 move, with and without
broadening, and a degenerate kept pair."""
import numpy as np
import pytest

from oracle import ctm_grad as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_08212_gb300 import ctm as C
    C.load()
    return C


def _check(ctm, U, s, Vt, gU, eps):
    import torch
    ref = G.svd_left_adjoint(*(torch.tensor(x) for x in (U, s, Vt, gU)), eps).numpy()
    rc, gM = ctm.ctm_svd_left_adjoint(U, s, Vt, gU, eps)
    torch.cuda.synchronize()
    assert rc == ctm.OK
    got = gM.cpu().numpy()
    assert np.all(np.isfinite(got))
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


CASES = [((12, 7), 3), ((6, 10), 4), ((9, 9), 5), ((300, 200), 37), ((2048, 272), 256),
         ((272, 2048), 200), ((1, 5), 1)]


@pytest.mark.parametrize("shape,k", CASES)
@pytest.mark.parametrize("eps", [0.0, 1e-12])
def test_svd_left_adjoint_matches_oracle(ctm, shape, k, eps):
    rng = np.random.default_rng(shape[0] * 1000 + shape[1] + k)
    U, s, Vt = np.linalg.svd(rng.standard_normal(shape), full_matrices=False)
    _check(ctm, U, s, Vt, rng.standard_normal((shape[0], k)), eps)


def test_degenerate_kept_pair(ctm):
    rng = np.random.default_rng(11)
    Q1, _ = np.linalg.qr(rng.standard_normal((8, 5)))
    Q2, _ = np.linalg.qr(rng.standard_normal((5, 5)))
    s = np.array([3.0, 2.0, 2.0, 1.0, 0.5])
    _check(ctm, Q1, s, Q2.T, rng.standard_normal((8, 3)), 1e-12)


def test_bad_arguments(ctm):
    U, s, Vt = np.linalg.svd(np.random.default_rng(0).standard_normal((6, 4)), full_matrices=False)
    rc, _ = ctm.ctm_svd_left_adjoint(U, s, Vt, np.zeros((6, 5)), 1e-12)  # k > r
    assert rc == ctm.ERR_ARG
    rc, _ = ctm.ctm_svd_left_adjoint(U, s, Vt, np.zeros((6, 2)), -1.0)  # eps < 0
    assert rc == ctm.ERR_ARG


@pytest.mark.parametrize("eps", [0.0, 1e-12])
def test_rank_deficient_tall_matrix(ctm, eps):
    """A tall 40 x 12 matrix of rank 7 with k = 10 kept columns: three kept
    singular values are zero (and exactly degenerate with each other).  Both
    sides take the pseudo-inverse convention; the result is finite and equal."""
    rng = np.random.default_rng(5)
    X = rng.standard_normal((40, 7)) @ rng.standard_normal((7, 12))
    U, s, Vt = np.linalg.svd(X, full_matrices=False)
    s[7:] = 0.0  # exact zeros (LAPACK returns ~1e-15 there)
    _check(ctm, U, s, Vt, rng.standard_normal((40, 10)), eps)


def test_zero_matrix(ctm):
    """s = 0 everywhere: every term takes the zero convention, gM = 0."""
    _check(ctm, np.eye(5)[:, :3], np.zeros(3), np.eye(3), np.ones((5, 2)), 0.0)
