"""Pins of the gradient oracle (oracle/ctm_grad.py) against facts outside it.

* Its forward pass is the (separately pinned) numpy oracle's reduced-sequential
  iteration: same energy to 1e-12.
* The hand-written adjoint of the truncated SVD equals central finite
  differences and PyTorch's own SVD backward on gauge-invariant functions of the
  kept left vectors, for tall and wide matrices, and stays finite and correct
  when kept singular values are degenerate (the Lorentzian broadening).
* The gradient of the energy after CTM iterations equals central finite
  differences (h = 1e-6) of the numpy oracle's energy on 64 entries of A and B,
  with and without checkpointed iterations.
* The hand-written reverse pass of the sequential absorption (pairwise
  contractions of the incoming gradient) equals autograd for every input.

The exactness pins run the adjoint with a vanishing broadening (EXACT): the
Lorentzian term shifts every pair whose squared relative gap is near eps, and
the spectra of a CTM move have such pairs among small kept values.  The
broadened adjoint (eps = 1e-12 relative to s_max^4) is pinned on degenerate
spectra, where the exact one divides by zero, and its bias on the energy
gradient is bounded.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ctm_grad as G  # noqa: E402
from oracle import ctm_oracle as O  # noqa: E402
from paper_2306_08212_gb300 import inputs as I  # noqa: E402

EXACT = 1e-40  # broadening small enough to leave every non-degenerate pair exact


def _np_energy(env0, A, B, chi, iters):
    env = {k: v.copy() for k, v in env0.items()}
    for _ in range(iters):
        for d in O.MOVE_ORDER:
            O.move(env, d, A, B, chi, chi, "reduced_sequential")
    H = O.heisenberg_bond()
    return float(np.mean([O.expect_bond(env, A, B, b, H) for b in range(4)]))


def _setup(D=2, chi=6, seed=3):
    A, B = I.random_sites(2, D, seed)
    env0 = O.init_env(A, B, chi)
    return A, B, env0


def test_forward_is_the_numpy_oracle():
    A, B, env0 = _setup()
    for iters in (1, 2):
        e_np = _np_energy(env0, A, B, 6, iters)
        e_t = float(G.energy(env0, torch.tensor(A), torch.tensor(B), 6, iters))
        assert abs(e_t - e_np) < 1e-12


def _projector_loss(Uk, W):
    return torch.sum(W * (Uk @ Uk.T))  # depends on span(Uk) only


@pytest.mark.parametrize("shape,k", [((12, 7), 3), ((6, 10), 4), ((9, 9), 5)])
def test_truncated_svd_adjoint(shape, k):
    rng = np.random.default_rng(7)
    M0 = rng.standard_normal(shape)
    W = torch.tensor(rng.standard_normal((shape[0], shape[0])))
    M = torch.tensor(M0, requires_grad=True)
    g = torch.autograd.grad(_projector_loss(G.TruncatedLeft.apply(M, k, EXACT), W), M)[0].numpy()
    # PyTorch's own SVD backward (non-degenerate spectrum)
    M2 = torch.tensor(M0, requires_grad=True)
    U = torch.linalg.svd(M2, full_matrices=False)[0][:, :k]
    g_lib = torch.autograd.grad(_projector_loss(U, W), M2)[0].numpy()
    np.testing.assert_allclose(g, g_lib, rtol=0, atol=1e-10 * np.abs(g_lib).max())
    # central differences
    h = 1e-6
    fd = np.zeros_like(M0)
    for i in range(shape[0]):
        for j in range(shape[1]):
            Mp, Mm = M0.copy(), M0.copy()
            Mp[i, j] += h
            Mm[i, j] -= h
            fp = _projector_loss(G.TruncatedLeft.apply(torch.tensor(Mp), k, EXACT), W)
            fm = _projector_loss(G.TruncatedLeft.apply(torch.tensor(Mm), k, EXACT), W)
            fd[i, j] = float(fp - fm) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=0, atol=1e-7 * np.abs(fd).max())


def test_degenerate_kept_singular_values():
    """s = (3, 2, 2, 1, 0.5) with k = 3: the kept pair is degenerate, the cut is not.
    The projector onto the kept span is smooth, its gradient finite; F without
    broadening would divide by zero."""
    rng = np.random.default_rng(11)
    Q1, _ = np.linalg.qr(rng.standard_normal((8, 5)))
    Q2, _ = np.linalg.qr(rng.standard_normal((5, 5)))
    M0 = Q1 @ np.diag([3.0, 2.0, 2.0, 1.0, 0.5]) @ Q2.T
    W = torch.tensor(rng.standard_normal((8, 8)))
    M = torch.tensor(M0, requires_grad=True)
    g = torch.autograd.grad(_projector_loss(G.TruncatedLeft.apply(M, 3, 1e-12), W), M)[0].numpy()
    assert np.all(np.isfinite(g))
    h = 1e-6
    fd = np.zeros_like(M0)
    for i in range(8):
        for j in range(5):
            Mp, Mm = M0.copy(), M0.copy()
            Mp[i, j] += h
            Mm[i, j] -= h
            fp = _projector_loss(G.TruncatedLeft.apply(torch.tensor(Mp), 3, 1e-12), W)
            fm = _projector_loss(G.TruncatedLeft.apply(torch.tensor(Mm), 3, 1e-12), W)
            fd[i, j] = float(fp - fm) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=0, atol=1e-6 * np.abs(fd).max())


def test_rank_deficient_kept_columns_pseudo_inverse():
    """M of rank 7 (40 x 12), k = 10 kept columns, three of them with s = 0.  A loss
    that depends only on the seven columns with s > 0 (sign-invariant: sum of
    c_ij u_ij^2) has a well-defined gradient; the adjoint with the zero conventions
    (F_ij = 0 for the degenerate zero pair, pseudo-inverse 0 for s = 0) equals its
    central differences, where a plain 1/s or 1/(s_j^2 - s_i^2) gives NaN."""
    rng = np.random.default_rng(5)
    M0 = rng.standard_normal((40, 7)) @ rng.standard_normal((7, 12))
    c = rng.standard_normal((40, 7))

    def loss(M):
        U = np.linalg.svd(M, full_matrices=False)[0]
        return float(np.sum(c * U[:, :7] ** 2))

    U, s, Vt = np.linalg.svd(M0, full_matrices=False)
    s[7:] = 0.0
    gU = np.zeros((40, 10))
    gU[:, :7] = 2 * c * U[:, :7]
    for eps in (0.0, 1e-12):
        g = G.svd_left_adjoint(*(torch.tensor(x) for x in (U, s, Vt, gU)), eps).numpy()
        assert np.all(np.isfinite(g))
        if eps == 0.0:
            h = 1e-6
            fd = np.zeros_like(M0)
            for idx in np.ndindex(M0.shape):
                Mp, Mm = M0.copy(), M0.copy()
                Mp[idx] += h
                Mm[idx] -= h
                fd[idx] = (loss(Mp) - loss(Mm)) / (2 * h)
            np.testing.assert_allclose(g, fd, rtol=0, atol=1e-6 * np.abs(fd).max())


def test_energy_gradient_matches_central_differences():
    """D=2, chi=6: all 32 entries of A and all 32 of B (64 in total), one iteration."""
    A, B, env0 = _setup()
    chi, iters = 6, 1
    _, gA, gB = G.energy_and_grad(env0, A, B, chi, iters, eps=EXACT)
    h = 1e-6
    for X, g, which in ((A, gA, "A"), (B, gB, "B")):
        fd = np.zeros_like(X)
        for idx in np.ndindex(X.shape):
            Xp, Xm = X.copy(), X.copy()
            Xp[idx] += h
            Xm[idx] -= h
            if which == "A":
                ep, em = _np_energy(env0, Xp, B, chi, iters), _np_energy(env0, Xm, B, chi, iters)
            else:
                ep, em = _np_energy(env0, A, Xp, chi, iters), _np_energy(env0, A, Xm, chi, iters)
            fd[idx] = (ep - em) / (2 * h)
        np.testing.assert_allclose(g, fd, rtol=0, atol=1e-6 * np.abs(fd).max())
    # the energy does not change when A is scaled, so dE/dA is orthogonal to A
    assert abs(np.sum(gA * A)) < 1e-9 * np.abs(gA).max()


def test_broadened_energy_gradient_stays_close():
    """With eps = 1e-12 the energy gradient differs from the exact one only through
    pairs of kept singular values whose squared relative gap is near eps."""
    A, B, env0 = _setup()
    _, gA0, gB0 = G.energy_and_grad(env0, A, B, 6, 1, eps=EXACT)
    _, gA1, gB1 = G.energy_and_grad(env0, A, B, 6, 1, eps=1e-12)
    assert np.all(np.isfinite(gA1)) and np.all(np.isfinite(gB1))
    scale = max(np.abs(gA0).max(), np.abs(gB0).max())
    assert max(np.abs(gA1 - gA0).max(), np.abs(gB1 - gB0).max()) < 5e-2 * scale


def test_checkpointed_iterations_give_the_same_gradient():
    """Checkpointing each CTM iteration (only its output environment kept, the rest
    recomputed in the backward pass) changes memory, not the gradient."""
    A, B, env0 = _setup()
    e0, gA0, gB0 = G.energy_and_grad(env0, A, B, 6, 2, eps=EXACT)
    e1, gA1, gB1 = G.energy_and_grad(env0, A, B, 6, 2, eps=EXACT, checkpoint=True)
    assert e1 == e0
    np.testing.assert_allclose(gA1, gA0, rtol=0, atol=1e-13 * np.abs(gA0).max())
    np.testing.assert_allclose(gB1, gB0, rtol=0, atol=1e-13 * np.abs(gB0).max())


def test_hand_written_absorption_adjoint_equals_autograd():
    """The reverse pass of the six sequential contractions (Fig. 4b), written out as
    pairwise contractions of the incoming gradient, equals PyTorch's autograd of the
    forward, for every input (T, the site used twice, and the four isometry halves)."""
    rng = np.random.default_rng(5)
    d, D, chi, c = 2, 3, 5, 4
    shapes = [(chi, D, D, chi), (d, D, D, D, D), (chi, D, c), (c, D, chi), (chi, D, c), (c, D, chi)]
    xs = [torch.tensor(rng.standard_normal(sh), requires_grad=True) for sh in shapes]
    out = G.absorb_edge_seq(*xs)
    g = torch.tensor(rng.standard_normal(out.shape))
    ref = torch.autograd.grad(out, xs, g)
    got = G.absorb_edge_seq_adjoint(*(x.detach() for x in xs), g)
    for r, h in zip(ref, got):
        np.testing.assert_allclose(h.numpy(), r.numpy(), rtol=0, atol=1e-12 * np.abs(r.numpy()).max())
    # each use of the site contributes: the ket use alone is not the gradient
    sp = G.ABSORB_SEQ_SPECS
    X1 = G.ein(sp[0], xs[0].detach(), xs[4].detach())
    X2 = G.ein(sp[1], X1, xs[1].detach())
    X3 = G.ein(sp[2], X2, xs[2].detach())
    X4 = G.ein(sp[3], X3, xs[5].detach())
    gX5, _ = G.contract_adjoint(sp[5], G.ein(sp[4], X4, xs[1].detach()), xs[3].detach(), g)
    _, gS_bra = G.contract_adjoint(sp[4], X4, xs[1].detach(), gX5)
    assert np.abs((got[1] - gS_bra).numpy()).max() > 1e-3 * np.abs(ref[1].numpy()).max()
