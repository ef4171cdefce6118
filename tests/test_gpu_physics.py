"""GPU runs checked against exact results and invariants rather than the oracle.

* Ising-norm PEPS (D=2 per layer): ln Z per site (Onsager), nearest-neighbour
  <s s'> and the magnetisation (Yang), every mode, through ctm_converge.
* Full-size workload of the bench (d=2, D=8, chi=256) in mixed precision: the
  spectra are descending, non-negative and normalised, energies lie in the
  spectrum of S.S, and BF16 agrees with TF32 to the BF16 error level.
"""
import numpy as np
import pytest

from oracle import ctm_oracle as O
from oracle import onsager as ON
from paper_2306_08212_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_08212_gb300 import ctm as C
    C.load()
    return C


SZ = np.diag([1.0, -1.0])


@pytest.mark.parametrize("mode", ["standard", "reduced_env", "reduced_sequential"])
@pytest.mark.parametrize("beta,plus,tol_lnz,tol_nn", [(0.40, False, 2e-6, 2e-4),
                                                     (0.48, True, 2e-6, 2e-4),
                                                     (0.44, False, 5e-4, 2e-2)])
def test_ising_norm_peps_matches_onsager(ctm, mode, beta, plus, tol_lnz, tol_nn):
    A, W = I.ising_peps(beta)
    bnd = np.outer(W[0], W[0]) if plus else None
    g = ctm.Env(A, A, 16, boundary=bnd)
    try:
        g.converge(mode, max_iter=40, tol=1e-12)
        lnz = g.log_kappa()
        nn = g.expect_bond(0, np.kron(SZ, SZ))
        m = g.expect_bond(0, np.kron(SZ, np.eye(2)))
        assert abs(lnz - ON.lnz_single_integral(beta)) < tol_lnz
        assert abs(nn - ON.nn_correlation(beta)) < tol_nn
        assert abs(abs(m) - ON.magnetization(beta)) < max(tol_nn, 2e-4 if plus else 1e-8)
        # the four bonds are equivalent for this uniform state
        for b in range(1, 4):
            assert abs(g.expect_bond(b, np.kron(SZ, SZ)) - nn) < tol_nn
    finally:
        g.free()


def _spectra_ok(spectra):
    for s in spectra:
        assert np.all(np.isfinite(s)) and np.all(s >= 0)
        assert np.all(np.diff(s) <= 1e-15)
        assert abs(np.sum(s * s) - 1.0) < 1e-12


def test_full_size_bench_workload_properties(ctm):
    A, B = I.random_sites(2, 8, 0)
    H = O.heisenberg_bond()
    out = {}
    for prec in ("tf32", "bf16"):
        g = ctm.Env(A, B, 256, precision=prec)
        try:
            for d in O.MOVE_ORDER:
                g.move(d, "reduced_sequential")
            spec = g.corner_spectra()
            _spectra_ok(spec)
            assert all(len(s) == 256 for s in spec)
            en = [g.expect_bond(b, H) for b in range(4)]
            assert all(-0.75 - 1e-9 <= e <= 0.25 + 1e-9 for e in en)
            assert np.isfinite(g.log_kappa())
            out[prec] = (en, spec)
        finally:
            g.free()
    de = max(abs(a - b) for a, b in zip(out["tf32"][0], out["bf16"][0]))
    ds = max(np.abs(a[:32] - b[:32]).max() for a, b in zip(out["tf32"][1], out["bf16"][1]))
    print(f"D=8 chi=256: |E_bf16 - E_tf32| = {de:.3e}, top-32 spectra {ds:.3e}")
    assert de < 1e-2 and ds < 5e-2


def _product_env(D, c0, seed):
    """Environment whose every tensor is a ket copy times a bra copy, at chi = c0^2
    (legs fused ket-slow): C = c (x) c, T = t (x) t.  The bond density matrix of the
    window is then n n^T with n the ket-only window, so the bond energy has an exact
    value computed from the small chi = c0 tensors alone."""
    rng = np.random.default_rng(seed)
    small, env = {}, {}
    for k in range(1, 5):
        for x in "ab":
            c = rng.standard_normal((c0, c0))
            t = rng.standard_normal((c0, D, c0))
            c, t = c / np.linalg.norm(c), t / np.linalg.norm(t)
            small[("C", k, x)], small[("T", k, x)] = c, t
            env[("C", k, x)] = np.einsum("ab,AB->aAbB", c, c).reshape(c0 * c0, c0 * c0)
            env[("T", k, x)] = np.einsum("akb,AKB->aAkKbB", t, t).reshape(c0 * c0, D, D, c0 * c0)
    return small, env


def _ket_window(s, A, B):
    """n[p, q]: the 2 x 4 window of the horizontal a-b bond with the ket layer only
    (corners [prev, next], edges [prev, ket, next] clockwise; site (p, u, l, d, r)),
    contracted pairwise column by column."""
    e = np.einsum
    L = e("dg,gue->due", s[("C", 1, "a")], s[("T", 2, "a")])
    L = e("due,mld->mlue", L, s[("T", 1, "a")])
    L = e("mlue,pulnr->mepnr", L, A)
    L = e("mepnr,om->epnro", L, s[("C", 4, "a")])
    L = e("epnro,kno->eprk", L, s[("T", 4, "a")])
    R = e("ewz,zh->ewh", s[("T", 2, "b")], s[("C", 2, "b")])
    R = e("ewh,hvt->ewvt", R, s[("T", 3, "b")])
    R = e("ewvt,qwryv->etqry", R, B)
    R = e("etqry,ti->eqryi", R, s[("C", 3, "b")])
    R = e("eqryi,iyk->eqrk", R, s[("T", 4, "b")])
    return e("eprk,eqrk->pq", L, R)


def test_single_large_instance_d10_chi400(ctm):
    """Single large instance, D=10, chi=400, reduced-sequential in BF16.

    With a ket (x) bra product environment at chi = 20^2 the bond energy of the
    sequential density matrix (largest intermediate chi^2 d^2 D^4 = 51 GB here) has an
    exact value from the chi = 20 ket window; it must match to 1e-9.  Then, from a seeded
    random environment at full chi (growing the folded one with standard moves would
    take the O(chi^3 D^6) path this mode avoids), one warm and one timed iteration of
    moves: the corner spectra stay full length, sorted and unit-normalised."""
    import time

    import torch
    D, c0 = 10, 20
    chi = c0 * c0
    A, B = I.random_sites(2, D, 0)
    small, env = _product_env(D, c0, seed=2)
    n = _ket_window(small, A, B).reshape(-1)
    H = O.heisenberg_bond()
    e_exact = float(n @ H @ n / (n @ n))
    g = ctm.Env(A, B, chi, precision=ctm.BF16 | ctm.INIT_NO_GROW)
    try:
        for (kind, k, x), v in env.items():
            g.set_tensor(0 if kind == "C" else 1, k, 0 if x == "a" else 1, v)
        e = g.expect_bond(0, H)
        print(f"D=10 chi=400 product environment: E_bond = {e:.12f}, exact {e_exact:.12f}")
        assert abs(e - e_exact) < 1e-9
        for (kind, k, x), v in I.random_env_tensors(D, chi, seed=2).items():
            g.set_tensor(0 if kind == "C" else 1, k, 0 if x == "a" else 1, v)
        for d in O.MOVE_ORDER:
            g.move(d, "reduced_sequential")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for d in O.MOVE_ORDER:
            g.move(d, "reduced_sequential")
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        spec = g.corner_spectra()
        _spectra_ok(spec)
        assert all(len(s) == chi for s in spec)
        print(f"D=10 chi=400 bf16 reduced-sequential: {4 / dt:.2f} moves/s")
    finally:
        g.free()
