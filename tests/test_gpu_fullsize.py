"""GPU parity where the projector factorisations take their large-size paths, and the
errors of the mixed-precision modes stated against FP64.

* The truncated SVD itself (``ctm_truncated_svd_test``): exact Jacobi and the
  randomized subspace iteration run to convergence, against LAPACK, on matrices
  with a decaying spectrum (the shape of every CTM projector problem), compared as
  subspaces (RMS sine of the principal angles).
* FP64 reduced-sequential moves with factorisations of n = chi D = 1200 (D=3,
  chi=400) and n = 2048 (D=8, chi=256, the size of the bench) against the oracle:
  both above the exact-Jacobi limit (1024), so on the randomized path.
* FP64 standard moves with n = chi D^2 = 768 (exact Jacobi) and 1280 (randomized)
  on environments grown from the fold by both sides (D=4).
* TF32 and BF16 errors against the oracle at D=6, chi=144 and against the FP64 path
  (itself pinned above) at D=8, chi=256 after four iterations.

Gauge-invariant outputs only: the 8 corner spectra, the spectra of the 8 edges
reshaped as (prev) x (ket, bra, next) and (prev, ket, bra) x (next) (an isometry
changes an edge only by orthogonal maps on its bond legs), bond energies and ln kappa.
Inputs: seeded random sites (N(0,1), unit norm) and seeded positive random
environments (sums of two ket (x) bra products, chi = c0^2): a positive boundary
keeps ln kappa and the energies physical, and two terms break the Kronecker
degeneracies of a single product.  At D=8 the bond legs carry weights exp(-0.3 i)
so that the spectra decay as a converged environment's do (a flat random spectrum
leaves the truncation at the cut determined only to ~1e-9).
"""
import time

import numpy as np
import pytest

from oracle import ctm_oracle as O
from paper_2306_08212_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def ctm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_08212_gb300 import ctm as C
    C.load()
    return C


def _unit_sv(X):
    s = np.linalg.svd(X, compute_uv=False)
    return s / np.linalg.norm(s)


def _invariants(get):
    """Corner spectra and edge spectra (two reshapes) of an environment given by
    get(kind, k, x) -> ndarray."""
    out = {}
    for k in range(1, 5):
        for x in "ab":
            C = get("C", k, x)
            out[("C", k, x)] = _unit_sv(C)
            T = get("T", k, x)
            out[("T<", k, x)] = _unit_sv(T.reshape(T.shape[0], -1))
            out[("T>", k, x)] = _unit_sv(T.reshape(-1, T.shape[3]))
    return out


def _gpu_getter(g):
    return lambda kind, k, x: g.tensor(0 if kind == "C" else 1, k, 0 if x == "a" else 1)


def _max_gap(a, b, n=None):
    gaps = []
    for key in a:
        x, y = a[key], b[key]
        m = max(len(x), len(y)) if n is None else n
        u = np.zeros(m); u[: min(m, len(x))] = x[:m]
        v = np.zeros(m); v[: min(m, len(y))] = y[:m]
        gaps.append(np.abs(u - v).max())
    return max(gaps)


def _set_env(g, env):
    for (kind, k, x), v in env.items():
        g.set_tensor(0 if kind == "C" else 1, k, 0 if x == "a" else 1, v)


def _span_gap(U, V):
    """RMS sine of the principal angles between span(U) and span(V)."""
    R = V - U @ (U.T @ V)
    return np.linalg.norm(R) / np.sqrt(U.shape[1])


def _decaying(rng, rows, cols, decades):
    r = min(rows, cols)
    U, _ = np.linalg.qr(rng.standard_normal((rows, r)))
    V, _ = np.linalg.qr(rng.standard_normal((cols, r)))
    s = 10.0 ** (-decades * np.arange(r) / r)
    return (U * s) @ V.T


@pytest.mark.parametrize("path,rows,cols,k", [(0, 2500, 2300, 256), (2, 1400, 1300, 200),
                                              (1, 1400, 1300, 200), (1, 300, 2100, 90),
                                              (0, 2048, 2048, 256), (2, 3000, 500, 300)])
def test_truncated_svd_paths_match_lapack(ctm, path, rows, cols, k):
    """path 0 above min side 1024 takes the randomized subspace iteration."""
    rng = np.random.default_rng(rows + cols + k)
    # six decades over the spectrum: the gap at the cut keeps the leading-k span
    # determined to ~1e-11 by FP64 data (it is only as sharp as u / relative gap)
    M = _decaying(rng, rows, cols, 6)
    rc, U = ctm.ctm_truncated_svd_test(path, M, k)
    assert rc == ctm.OK
    ref = np.linalg.svd(M, full_matrices=False)[0][:, :k]
    assert np.abs(U.T @ U - np.eye(k)).max() < 1e-12
    gap = _span_gap(ref, U)
    print(f"truncated SVD path {path} {rows}x{cols} k={k}: span gap {gap:.2e}")
    assert gap < TOL


def _compare_fp64(g, env, A, B, energies=True, lnk=True):
    inv_o = _invariants(lambda kind, k, x: env[(kind, k, x)])
    inv_g = _invariants(_gpu_getter(g))
    gap = _max_gap(inv_o, inv_g)
    out = {"spectra": gap}
    H = O.heisenberg_bond()
    if energies:
        bonds = range(4) if energies is True else energies
        out["energy"] = max(abs(O.expect_bond_seq(env, A, B, b, H) - g.expect_bond(b, H))
                            for b in bonds)
    if lnk:
        out["lnk"] = abs(O.log_kappa_sites(env, A, B) - g.log_kappa())
    return out


def test_fp64_reduced_sequential_d3_chi400_matches_oracle(ctm):
    """n = chi D = 1200: above the exact-Jacobi limit; left then up move."""
    D, c0 = 3, 20
    chi = c0 * c0
    A, B = I.random_sites(2, D, 3)
    env = I.positive_env_tensors(D, c0, seed=2)
    g = ctm.Env(A, B, chi, precision=ctm.FP64 | ctm.INIT_NO_GROW)
    try:
        _set_env(g, env)
        for d in ("left", "up"):
            O.move(env, d, A, B, chi, chi, "reduced_sequential")
            g.move(d, "reduced_sequential")
        gaps = _compare_fp64(g, env, A, B)
        print(f"FP64 reduced-sequential D=3 chi=400, 2 moves: {gaps}")
        assert all(v < TOL for v in gaps.values())
    finally:
        g.free()


def test_fp64_reduced_sequential_d8_chi256_matches_oracle(ctm):
    """The size of the bench: every v1 factorisation is 2048 x 2048."""
    D, c0 = 8, 16
    chi = c0 * c0
    A, B = I.random_sites(2, D, 0)
    env = I.positive_env_tensors(D, c0, seed=2, decay=0.3)
    g = ctm.Env(A, B, chi, precision=ctm.FP64 | ctm.INIT_NO_GROW)
    try:
        _set_env(g, env)
        t0 = time.perf_counter()
        O.move(env, "left", A, B, chi, chi, "reduced_sequential")
        t1 = time.perf_counter()
        g.move("left", "reduced_sequential")
        g.corner_spectrum(0)
        t2 = time.perf_counter()
        gaps = _compare_fp64(g, env, A, B, energies=[0], lnk=False)
        print(f"FP64 reduced-sequential D=8 chi=256, left move: {gaps} "
              f"(oracle {t1 - t0:.1f} s, GPU {t2 - t1:.1f} s)")
        assert all(v < TOL for v in gaps.values())
    finally:
        g.free()


@pytest.mark.parametrize("chi,moves", [(48, ("left", "up", "right", "down")), (80, ("left", "up"))])
def test_fp64_standard_grown_matches_oracle(ctm, chi, moves):
    """D=4: the standard projector factorises n = chi D^2 = 768 (exact Jacobi) and
    1280 (randomized subspace iteration) on environments grown from the fold."""
    D = 4
    A, B = I.random_sites(2, D, 4)
    env = O.init_env(A, B, chi)
    g = ctm.Env(A, B, chi, precision=ctm.FP64)
    try:
        gaps0 = _compare_fp64(g, env, A, B, energies=[0], lnk=False)
        for d in moves:
            O.move(env, d, A, B, chi, chi, "standard")
            g.move(d, "standard")
        gaps = _compare_fp64(g, env, A, B)
        print(f"FP64 standard D=4 chi={chi}: grown {gaps0}, after {len(moves)} moves {gaps}")
        assert all(v < TOL for v in gaps0.values())
        assert all(v < TOL for v in gaps.values())
    finally:
        g.free()


def _run(ctm, prec, A, B, chi, env, iters):
    g = ctm.Env(A, B, chi, precision=ctm.PRECISIONS[prec] | ctm.INIT_NO_GROW)
    try:
        _set_env(g, env)
        for _ in range(iters):
            for d in O.MOVE_ORDER:
                g.move(d, "reduced_sequential")
        H = O.heisenberg_bond()
        return ([g.expect_bond(b, H) for b in range(4)], _invariants(_gpu_getter(g)),
                g.log_kappa())
    finally:
        g.free()


def test_mixed_precision_errors_vs_oracle_d6_chi144(ctm):
    """D=6, chi=144 (random sites, seeded positive starting environment), two
    reduced-sequential iterations: FP64, TF32 and BF16 against the oracle."""
    D, c0, iters = 6, 12, 2
    chi = c0 * c0
    A, B = I.random_sites(2, D, 0)
    env0 = I.positive_env_tensors(D, c0, seed=2)
    env = {k: v.copy() for k, v in env0.items()}
    for _ in range(iters):
        for d in O.MOVE_ORDER:
            O.move(env, d, A, B, chi, chi, "reduced_sequential")
    H = O.heisenberg_bond()
    e_ref = [O.expect_bond_seq(env, A, B, b, H) for b in range(4)]
    inv_ref = _invariants(lambda kind, k, x: env[(kind, k, x)])
    lnk_ref = O.log_kappa_sites(env, A, B)
    bounds = {"fp64": 1e-8, "tf32": 1e-3, "bf16": 1e-2}
    for prec in ("fp64", "tf32", "bf16"):
        e, inv, lnk = _run(ctm, prec, A, B, chi, env0, iters)
        de = max(abs(a - b) for a, b in zip(e, e_ref))
        ds = _max_gap(inv_ref, inv, 32)
        dk = abs(lnk - lnk_ref)
        print(f"D=6 chi=144 {prec} vs oracle after {iters} iterations: |dE_bond| = {de:.3e}, "
              f"top-32 spectra {ds:.3e}, |d ln kappa| = {dk:.3e}")
        assert de < bounds[prec] and dk < bounds[prec] and ds < 10 * bounds[prec]


def test_mixed_precision_errors_vs_fp64_d8_chi256(ctm):
    """The bench size, four reduced-sequential iterations from one seeded positive
    environment in FP64 (pinned to the oracle above), TF32 and BF16."""
    D, c0, iters = 8, 16, 4
    chi = c0 * c0
    A, B = I.random_sites(2, D, 0)
    env0 = I.positive_env_tensors(D, c0, seed=2, decay=0.3)
    res = {}
    for prec in ("fp64", "tf32", "bf16"):
        t0 = time.perf_counter()
        res[prec] = _run(ctm, prec, A, B, chi, env0, iters)
        print(f"D=8 chi=256 {prec}: {iters} iterations + observables in "
              f"{time.perf_counter() - t0:.1f} s, E_bond = {res[prec][0]}")
    e0, inv0, k0 = res["fp64"]
    for prec, bound in (("tf32", 1e-3), ("bf16", 1e-2)):
        e, inv, k = res[prec]
        de = max(abs(a - b) for a, b in zip(e, e0))
        ds = _max_gap(inv0, inv, 32)
        dk = abs(k - k0)
        print(f"D=8 chi=256 {prec} vs FP64 after {iters} iterations: |dE_bond| = {de:.3e}, "
              f"top-32 spectra {ds:.3e}, |d ln kappa| = {dk:.3e}")
        assert de < bound and dk < bound and ds < 10 * bound


def test_corner_spectra_preconditioned_match_lapack(ctm):
    """At D=8, chi=256 the corner spectra take an FP32 Jacobi run as a
    preconditioner (C V with V orthonormalised in FP64) before the FP64 Jacobi:
    the spectra before and after a move equal LAPACK's on the same corners."""
    D, c0 = 8, 16
    chi = c0 * c0
    A, B = I.random_sites(2, D, 0)
    env = I.positive_env_tensors(D, c0, seed=2, decay=0.3)
    g = ctm.Env(A, B, chi, precision=ctm.BF16 | ctm.INIT_NO_GROW)
    try:
        _set_env(g, env)

        def check(label):
            got = g.corner_spectra()
            gap = 0.0
            for i, s in enumerate(got):
                C = g.tensor(0, i // 2 + 1, i % 2)
                ref = _unit_sv(C)
                n = max(len(ref), len(s))
                u = np.zeros(n); u[: len(ref)] = ref
                v = np.zeros(n); v[: len(s)] = s
                gap = max(gap, np.abs(u - v).max())
            print(f"corner spectra ({label}) vs LAPACK: {gap:.2e}")
            assert gap < 1e-12

        check("positive environment")
        g.move("left", "reduced_sequential")
        check("after a move")
    finally:
        g.free()
