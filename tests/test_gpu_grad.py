"""GPU reverse pass (ctm_energy_grad, the torch.autograd.Function on top of it)
against the gradient oracle (oracle/ctm_grad.py, pinned on the CPU by central
differences of the numpy oracle) and against central differences of the GPU's
own energy.

The loss is the mean Heisenberg bond energy after `iters` reduced-sequential
iterations from a fixed starting environment; inputs are seeded random sites and
seeded positive environments (sums of two ket (x) bra products).  The exact
comparisons use a vanishing broadening (1e-40), as the oracle's pins do."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ctm_grad as G  # noqa: E402
from oracle import ctm_oracle as O  # noqa: E402
from paper_2306_08212_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu

EXACT = 1e-40


@pytest.fixture(scope="module")
def ctm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_08212_gb300 import ctm as C
    C.load()
    return C


def _env(ctm, A, B, env0, chi):
    g = ctm.Env(A, B, chi, precision=ctm.FP64 | ctm.INIT_NO_GROW)
    for (kind, k, x), v in env0.items():
        g.set_tensor(0 if kind == "C" else 1, k, 0 if x == "a" else 1, v)
    return g


@pytest.mark.parametrize("D,c0,iters", [(2, 3, 1), (2, 3, 2), (3, 3, 1)])
def test_energy_gradient_matches_oracle(ctm, D, c0, iters):
    chi = c0 * c0
    A, B = I.random_sites(2, D, 5)
    env0 = I.positive_env_tensors(D, c0, seed=4)
    E_ref, gA_ref, gB_ref = G.energy_and_grad(env0, A, B, chi, iters, eps=EXACT)
    g = _env(ctm, A, B, env0, chi)
    try:
        before = g.tensor(0, 1, 0)
        E, gA, gB = g.energy_grad(iters, O.heisenberg_bond(), EXACT)
        after = g.tensor(0, 1, 0)
    finally:
        g.free()
    scale = max(np.abs(gA_ref).max(), np.abs(gB_ref).max())
    dA, dB = np.abs(gA - gA_ref).max(), np.abs(gB - gB_ref).max()
    print(f"D={D} chi={chi} iters={iters}: E {E:.12f} (oracle {E_ref:.12f}), "
          f"|dgA| {dA:.2e} |dgB| {dB:.2e} of max |g| {scale:.2e}")
    assert abs(E - E_ref) < 1e-12
    assert dA < 1e-9 * scale and dB < 1e-9 * scale
    np.testing.assert_array_equal(before, after)  # the starting environment is held fixed


def test_energy_gradient_matches_central_differences_on_the_gpu(ctm):
    """32 random entries of A and B, h = 1e-6, energies from the GPU alone."""
    D, c0, iters = 3, 3, 2
    chi = c0 * c0
    A, B = I.random_sites(2, D, 6)
    env0 = I.positive_env_tensors(D, c0, seed=7)
    H = O.heisenberg_bond()
    g = _env(ctm, A, B, env0, chi)
    try:
        _, gA, gB = g.energy_grad(iters, H, EXACT)
        rng = np.random.default_rng(8)
        h = 1e-6
        for which, X, gX in (("A", A, gA), ("B", B, gB)):
            for flat in rng.choice(X.size, 16, replace=False):
                idx = np.unravel_index(flat, X.shape)
                vals = []
                for sgn in (1, -1):
                    Xp = X.copy()
                    Xp[idx] += sgn * h
                    g.set_sites(Xp, B) if which == "A" else g.set_sites(A, Xp)
                    vals.append(g.energy_grad(iters, H, EXACT)[0])
                fd = (vals[0] - vals[1]) / (2 * h)
                assert abs(fd - gX[idx]) < 1e-6 * max(np.abs(gA).max(), np.abs(gB).max()), (
                    which, idx, fd, gX[idx])
        g.set_sites(A, B)
    finally:
        g.free()


def test_autograd_function(ctm):
    """torch.autograd through ctm_energy gives the library's gradient, scaled by the
    incoming gradient."""
    D, c0, iters = 2, 3, 1
    chi = c0 * c0
    A, B = I.random_sites(2, D, 9)
    env0 = I.positive_env_tensors(D, c0, seed=10)
    H = O.heisenberg_bond()
    g = _env(ctm, A, B, env0, chi)
    try:
        At = torch.tensor(A, requires_grad=True)
        Bt = torch.tensor(B, requires_grad=True)
        E = ctm.ctm_energy(At, Bt, g, iters, H, EXACT)
        (3.0 * E).backward()
        E2, gA, gB = g.energy_grad(iters, H, EXACT)
        assert abs(float(E) - E2) < 1e-14
        np.testing.assert_allclose(At.grad.numpy(), 3.0 * gA, rtol=0, atol=1e-14)
        np.testing.assert_allclose(Bt.grad.numpy(), 3.0 * gB, rtol=0, atol=1e-14)
    finally:
        g.free()
