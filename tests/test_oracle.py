"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* Exact (untruncated) moves reproduce brute-force finite-lattice density
  matrices, in both modes and all four directions (Sec. II: a move absorbs a
  column; with chi large no projector truncates).
* The sequential ket-then-bra absorption with split isometries equals the
  double-layer absorption with the composed 4-index isometry (Sec. IV: the
  sequential order only re-brackets v = v^1 v^2).
* D = 1 product states: <S.S> factorises exactly, in both modes.
* The Ising-norm PEPS reproduces Onsager's free energy and nearest-neighbour
  correlation and Yang's magnetisation.
* Four quarter turns of a site are the identity.
* With v_l, v_r keeping the whole range of their boundary columns, the one-row
  reduced network equals the reduced-environment network written out as one
  einsum (Sec. III, Appendix).
"""
import numpy as np
import pytest

from oracle import ctm_oracle as O
from oracle import onsager as ON
from paper_2306_08212_gb300 import inputs as I
from tests import brute


HUGE = 10 ** 6  # a bond dimension that never truncates


def _iso(rng, m, n):
    q, _ = np.linalg.qr(rng.standard_normal((m, n)))
    return q


def test_rotation_four_quarter_turns_is_identity():
    A, _ = I.random_sites(2, 3, 5)
    assert np.array_equal(O.rotate_site(A, 4), A)
    # one quarter turn moves the up leg to the left slot
    R = O.rotate_site(A, 1)
    assert np.array_equal(R[:, 1, 2, 0, 1], A[:, 2, 0, 1, 1])


def test_sequential_absorption_equals_double_layer_with_composed_isometries():
    rng = np.random.default_rng(3)
    d, D, chi, chip = 2, 3, 5, 4
    T = rng.standard_normal((chi, D, D, chi))
    A = rng.standard_normal((d, D, D, D, D))
    S = O.edge_site_T1(A)
    vp1 = _iso(rng, chi * D, chip).reshape(chi, D, chip)
    vp2 = _iso(rng, chip * D, chi).reshape(chip, D, chi)
    vn1 = _iso(rng, chi * D, chip).reshape(chi, D, chip)
    vn2 = _iso(rng, chip * D, chi).reshape(chip, D, chi)
    seq = O.absorb_edge_seq(T, S, vp1, vp2, vn1, vn2)
    dbl = O.absorb_edge_double(T, S, O.compose(vp1, vp2), O.compose(vn1, vn2))
    assert seq.shape == (chi, D, D, chi)
    np.testing.assert_allclose(seq, dbl, rtol=0, atol=1e-13 * np.abs(dbl).max())


def test_sequential_absorption_checks_every_leg():
    """A planted transposition (prev <-> next projector) must break the equality."""
    rng = np.random.default_rng(4)
    d, D, chi = 2, 2, 3
    T = rng.standard_normal((chi, D, D, chi))
    A = rng.standard_normal((d, D, D, D, D))
    S = O.edge_site_T1(A)
    vs = [_iso(rng, chi * D, chi).reshape(chi, D, chi) for _ in range(4)]
    good = O.absorb_edge_double(T, S, O.compose(vs[0], vs[1]), O.compose(vs[2], vs[3]))
    bad = O.absorb_edge_seq(T, S, vs[2], vs[1], vs[0], vs[3])
    assert np.abs(good - bad).max() > 1e-3


def _env_fold(A, B):
    env = O.fold_init(A, B)
    return {k: O._normalize(v) for k, v in env.items()}


MODES = ["standard", "reduced_env", "reduced_sequential"]


@pytest.mark.parametrize("mode", MODES)
def test_fold_and_exact_moves_match_brute_force(mode):
    d, D = 2, 2
    A, B = I.random_sites(d, D, 11)
    env = _env_fold(A, B)
    # no move: each 1x2 window sits in a 3 x 4 patch
    # bond 0: a at (1,1); bond 1: b at (1,1)
    for bond, par in ((0, 0), (1, 1)):
        ref = brute.finite_rdm(A, B, 3, 4, ((1, 1), (1, 2)), a_parity=par)
        rho = O.bond_rdm(env, A, B, 0, "a" if bond == 0 else "b")
        np.testing.assert_allclose(rho / np.trace(rho), ref / np.trace(ref), atol=1e-13)
    # one exact left move adds two columns on the left, one exact right move
    # two on the right: a 3 x 8 patch with the pair at columns 3, 4
    O.move(env, "left", A, B, HUGE, HUGE, mode)
    O.move(env, "right", A, B, HUGE, HUGE, mode)
    for bond, par in ((0, 0), (1, 1)):
        ref = brute.finite_rdm(A, B, 3, 8, ((1, 3), (1, 4)), a_parity=par)
        rho = O.bond_rdm(env, A, B, 0, "a" if bond == 0 else "b")
        np.testing.assert_allclose(rho / np.trace(rho), ref / np.trace(ref), atol=1e-12)
        rho = O.bond_rdm_seq(env, A, B, 0, "a" if bond == 0 else "b")
        np.testing.assert_allclose(rho / np.trace(rho), ref / np.trace(ref), atol=1e-12)


@pytest.mark.parametrize("mode", MODES)
def test_exact_vertical_moves_match_brute_force(mode):
    d, D = 2, 2
    A, B = I.random_sites(d, D, 12)
    env = _env_fold(A, B)
    O.move(env, "up", A, B, HUGE, HUGE, mode)
    O.move(env, "down", A, B, HUGE, HUGE, mode)
    # in the frame turned one quarter counter-clockwise the vertical pair is
    # horizontal and the up/down moves are left/right moves
    Ar, Br = O.rotate_site(A, 1), O.rotate_site(B, 1)
    for x, par in (("a", 0), ("b", 1)):
        ref = brute.finite_rdm(Ar, Br, 3, 8, ((1, 3), (1, 4)), a_parity=par)
        rho = O.bond_rdm(env, A, B, 1, x)
        np.testing.assert_allclose(rho / np.trace(rho), ref / np.trace(ref), atol=1e-12)
        rho = O.bond_rdm_seq(env, A, B, 1, x)
        np.testing.assert_allclose(rho / np.trace(rho), ref / np.trace(ref), atol=1e-12)


@pytest.mark.parametrize("mode", MODES)
def test_product_state_factorises(mode):
    pa = np.array([0.8, 0.6])
    pb = np.array([0.28, -0.96])
    A, B = I.product_sites(pa, pb)
    env = O.init_env(A, B, 4)
    O.converge(env, A, B, 4, 4, mode, max_iter=3)
    sx = np.array([[0, 1], [1, 0]]) / 2
    sz = np.array([[1, 0], [0, -1]]) / 2
    ma = np.array([pa @ sx @ pa, pa @ sz @ pa])
    mb = np.array([pb @ sx @ pb, pb @ sz @ pb])
    exact = float(ma @ mb)  # <Sy> vanishes for real spinors
    H = O.heisenberg_bond()
    for bond in range(4):
        assert abs(O.expect_bond(env, A, B, bond, H) - exact) < 1e-14


def test_neel_product_state_energy():
    A, B = I.neel_sites(1, eps=0.0)
    env = O.init_env(A, B, 4)
    O.converge(env, A, B, 4, 4, "reduced_sequential", max_iter=2)
    for bond in range(4):
        assert abs(O.expect_bond(env, A, B, bond, O.heisenberg_bond()) + 0.25) < 1e-15


@pytest.mark.parametrize("D,chi,seed", [(2, 6, 1), (3, 5, 2)])
def test_sequential_bond_rdm_equals_double_layer(D, chi, seed):
    """bond_rdm_seq (ket and bra layers in turn) and bond_rdm (open double layer) are
    the same contraction in two orders: equal on random environments for all four
    bonds, and a planted swap of a site's ket legs breaks the equality."""
    A, B = I.random_sites(2, D, seed)
    env = I.random_env_tensors(D, chi, seed=seed + 10)
    for bond in range(4):
        r, x = O.BONDS[bond]
        a, b = O.bond_rdm(env, A, B, r, x), O.bond_rdm_seq(env, A, B, r, x)
        np.testing.assert_allclose(b, a, rtol=0, atol=1e-13 * np.abs(a).max())
    Bbad = B.transpose(0, 2, 1, 3, 4)  # u and l exchanged on one site
    a = O.bond_rdm(env, A, Bbad, 0, "a")
    b = O.bond_rdm_seq(env, A, B, 0, "a")
    assert np.abs(a / np.trace(a) - b / np.trace(b)).max() > 1e-3


def test_heisenberg_bond_is_the_spin_half_exchange():
    """Pins the operator of Eq. 1 as read here (S = sigma/2, antiferromagnetic sign),
    including its Sy Sy term, which the real product and Neel states cannot see:
    * for two spins 1/2, S_i . S_j = P/2 - 1/4 with P the swap of the two sites;
    * its spectrum is {-3/4 (singlet), 1/4, 1/4, 1/4 (triplet)};
    * the singlet (|01> - |10>)/sqrt 2 has -3/4, and (|00> + |11>)/sqrt 2 and
      (|00> - |11>)/sqrt 2, whose energies differ in sign if Sy Sy does, both 1/4;
    * the Sy Sy part equals kron(sy, sy) built from the complex Pauli matrix."""
    H = O.heisenberg_bond()
    swap = np.zeros((4, 4))
    for i in range(2):
        for j in range(2):
            swap[2 * j + i, 2 * i + j] = 1.0
    np.testing.assert_allclose(H, swap / 2 - np.eye(4) / 4, rtol=0, atol=1e-15)
    np.testing.assert_allclose(np.linalg.eigvalsh(H), [-0.75, 0.25, 0.25, 0.25], rtol=0, atol=1e-15)
    singlet = np.array([0, 1, -1, 0]) / np.sqrt(2)
    np.testing.assert_allclose(H @ singlet, -0.75 * singlet, rtol=0, atol=1e-15)
    for v in (np.array([1, 0, 0, 1]) / np.sqrt(2), np.array([1, 0, 0, -1]) / np.sqrt(2)):
        np.testing.assert_allclose(H @ v, 0.25 * v, rtol=0, atol=1e-15)
    sy = np.array([[0, -1j], [1j, 0]]) / 2
    sx = np.array([[0, 1], [1, 0]]) / 2
    sz = np.diag([0.5, -0.5])
    yy = H - np.kron(sx, sx) - np.kron(sz, sz)
    np.testing.assert_allclose(yy, np.kron(sy, sy).real, rtol=0, atol=1e-15)
    assert np.abs(np.kron(sy, sy).imag).max() == 0.0


def test_onsager_closed_forms_agree_with_each_other():
    for beta in (0.40, 0.44, 0.48):
        assert abs(ON.lnz_double_integral(beta) - ON.lnz_single_integral(beta)) < 1e-12
        # <s s'> = (1/2) d(ln Z / N)/d beta: two bonds per site
        h = 1e-5
        der = (ON.lnz_single_integral(beta + h) - ON.lnz_single_integral(beta - h)) / (2 * h)
        assert abs(0.5 * der - ON.nn_correlation(beta)) < 1e-6


def test_onsager_golden_table():
    rows = np.loadtxt("tests/golden/onsager.txt", comments="#")
    for beta, lnz, nn, m in rows:
        assert abs(ON.lnz_single_integral(beta) - lnz) < 1e-12
        assert abs(ON.nn_correlation(beta) - nn) < 1e-12
        assert abs(ON.magnetization(beta) - m) < 1e-12


def _ising_run(beta, chi, mode, plus_boundary, iters):
    A, W = I.ising_peps(beta)
    bnd = np.outer(W[0], W[0]) if plus_boundary else None
    env = O.init_env(A, A, chi, bnd)
    O.converge(env, A, A, chi, chi, mode, max_iter=iters, tol=1e-13)
    sz = np.diag([1.0, -1.0])
    zz = O.expect_bond(env, A, A, 0, np.kron(sz, sz))
    m = O.expect_bond(env, A, A, 0, np.kron(sz, np.eye(2)))
    lk = O.log_kappa_sites(env, A, A)
    return lk, zz, m


@pytest.mark.parametrize("mode", MODES)
def test_ising_high_temperature_matches_onsager(mode):
    beta = 0.40
    lk, zz, m = _ising_run(beta, 16, mode, False, 60)
    assert abs(lk - ON.lnz_single_integral(beta)) < 2e-6
    assert abs(zz - ON.nn_correlation(beta)) < 2e-4
    assert abs(m) < 1e-10


@pytest.mark.parametrize("mode", MODES)
def test_ising_ordered_phase_matches_onsager_and_yang(mode):
    beta = 0.48
    lk, zz, m = _ising_run(beta, 16, mode, True, 60)
    assert abs(lk - ON.lnz_single_integral(beta)) < 2e-6
    assert abs(zz - ON.nn_correlation(beta)) < 2e-4
    assert abs(m - ON.magnetization(beta)) < 2e-4


def test_reduced_env_projector_is_the_standard_one_when_the_right_half_is_exact():
    """Sec. III: the right half {y, T2_y, C2_y, T3_y} of the standard network is
    what a right-move absorption turns into {C2_x, T3_x}.  After one exact
    (untruncated) right column absorption the reduced network is therefore the
    standard upper half of the previous environment with its columns regrouped,
    and both give the same projector v v^T."""
    A, B = I.random_sites(2, 2, 21)
    env0 = _env_fold(A, B)
    env1 = {k: v.copy() for k, v in env0.items()}
    sites2 = {"a": O.rotate_site(A, 2), "b": O.rotate_site(B, 2)}
    O.column_absorb(env1, 2, sites2, HUGE, HUGE, "standard")  # one right column, exact
    sites = {"a": A, "b": B}
    for chi in (4, 9):
        v_std = O.projector_standard(O.View(env0, 0), "a", sites, chi)
        v_red = O.projector_reduced_env(O.View(env1, 0), "a", sites, chi)
        assert v_std.shape == v_red.shape
        Ps = O.ein("akbx,KLMx->akbKLM", v_std, v_std)
        Pr = O.ein("akbx,KLMx->akbKLM", v_red, v_red)
        np.testing.assert_allclose(Pr, Ps, rtol=0, atol=1e-10)
    # and a planted mistake (x's right half taken from y) breaks it
    v_bad = O.projector_reduced_env(O.View(env1, 0), "b", {"a": B, "b": A}, 4)
    Pb = O.ein("akbx,KLMx->akbKLM", v_bad, v_bad)
    v_std = O.projector_standard(O.View(env0, 0), "a", sites, 4)
    Ps = O.ein("akbx,KLMx->akbKLM", v_std, v_std)
    assert np.abs(Pb - Ps).max() > 1e-3


def test_row_correlator_x1_is_the_bond_expectation():
    """The strip of two sites is the 1x2 window of the bond density matrix."""
    A, B = I.random_sites(2, 2, 31)
    env = O.init_env(A, B, 8)
    O.converge(env, A, B, 8, 8, "standard", max_iter=5)
    sz = np.diag([0.5, -0.5])
    sx = np.array([[0, 0.5], [0.5, 0]])
    S = O.row_correlator(env, A, B, sz, sx, 3)
    two = O.expect_bond(env, A, B, 0, np.kron(sz, sx))
    one_a = O.expect_bond(env, A, B, 0, np.kron(sz, np.eye(2)))
    one_b = O.expect_bond(env, A, B, 0, np.kron(np.eye(2), sx))
    assert abs(S[0] - (two - one_a * one_b)) < 1e-13


def test_row_correlator_vanishes_for_product_states():
    A, B = I.product_sites([0.8, 0.6], [0.28, -0.96])
    env = O.init_env(A, B, 4)
    sz = np.diag([0.5, -0.5])
    S = O.row_correlator(env, A, B, sz, sz, 5)
    assert np.all(np.abs(S) < 1e-15)


def test_ising_row_correlator_decays_and_starts_at_onsager():
    beta = 0.40
    A, W = I.ising_peps(beta)
    env = O.init_env(A, A, 16)
    O.converge(env, A, A, 16, 16, "standard", max_iter=40, tol=1e-13)
    sz = np.diag([1.0, -1.0])
    S = O.row_correlator(env, A, A, sz, sz, 8)
    assert abs(S[0] - ON.nn_correlation(beta)) < 2e-4   # m = 0 at beta < beta_c
    assert np.all(np.diff(S) < 0) and S[-1] > 0


def _reduced_env_network(env, A):
    """Q[alpha, X_ket, X_bra, beta] of Sec. III written out as one network: the
    upper-left quadrant {C1_a, T2_a, T1_a; A (ket), A (bra)} closed on the right by
    {C2_a, T3_a}, legs as documented (C1[down,right], C2[left,down],
    T[prev, ket, bra, next]; site (p, u, l, d, r))."""
    return np.einsum("dg,gUVe,aLMd,pULXR,pVMYS,ez,zRSw->aXYw",
                     env[("C", 1, "a")], env[("T", 2, "a")], env[("T", 1, "a")], A, A,
                     env[("C", 2, "a")], env[("T", 3, "a")], optimize=True)


@pytest.mark.parametrize("chi_env,chip", [(4, HUGE), (4, 8), (5, 15)])
def test_reduced_network_is_the_reduced_environment_when_v_l_v_r_keep_their_range(chi_env, chip):
    """Appendix, Fig. 8 and Fig. 3c: v_l, v_r only compress the left and right
    boundary columns.  When they keep the whole range of L = C1 T1 and R = C2 T3
    (chi' >= chi D, chi >= the environment's chi) the one-row network
    M = C'1 T'2 C'2 equals the reduced-environment network of Sec. III entry by
    entry, whatever basis the factorisations return."""
    D = 2 if chi_env == 4 else 3
    A, B = I.random_sites(2, D, 31)
    env = I.random_env_tensors(D, chi_env, seed=5)
    sites = {"a": A, "b": B}
    M = O.reduced_network(O.View(env, 0), "a", sites, chi_env, chip)
    Q = _reduced_env_network(env, A)
    assert M.shape == Q.shape
    np.testing.assert_allclose(M, Q, rtol=0, atol=1e-12 * np.abs(Q).max())
    # a planted mistake: the sites of the two sublattices exchanged
    Mb = O.reduced_network(O.View(env, 0), "a", {"a": B, "b": A}, chi_env, chip)
    assert np.abs(Mb - Q).max() > 1e-3 * np.abs(Q).max()


def test_neel_golden_file_is_the_oracle_run():
    """tests/golden/neel_d4_chi64_50it.txt comes from the oracle: its first two
    spectrum changes are reproduced (to the three digits stored)."""
    vals = {}
    with open("tests/golden/neel_d4_chi64_50it.txt") as f:
        for line in f:
            if not line.startswith("#") and line.strip():
                key, *rest = line.split()
                vals[key] = [float(x) for x in rest]
    A, B = I.neel_sites(4, eps=1e-2, seed=0)
    env = O.init_env(A, B, 64)
    spec = O.corner_spectra(env)
    for it in range(2):
        for d in O.MOVE_ORDER:
            O.move(env, d, A, B, 64, 64, "reduced_sequential")
        new = O.corner_spectra(env)
        assert abs(O.spectrum_delta(spec, new) - vals["deltas"][it]) <= 2e-3 * vals["deltas"][it]
        spec = new
    assert len(vals["deltas"]) == 50 and -0.2501 < vals["energy_mean"][0] < -0.2499
