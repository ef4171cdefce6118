"""Plain FP64 CPU oracle of the corner-transfer (CTM) move for a 2-site {A,B} iPEPS.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
Python binding) imports, links or calls this module; only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py`` may use it.  It shares no code with the CUDA path.

What it follows (Lan & Evenbly, "Reduced Contraction Costs of Corner-Transfer
Methods for PEPS"):

* Sec. II and Fig. 1: the ansatz A, B of dims (d, D, D, D, D) on a checkerboard,
  the double-layer tensors a = sum_p A A*, and the corner/edge environment.
* Sec. II and Fig. 2: the left move absorbs a column into the left boundary and
  truncates the grown bonds with projectors P = v v^T, where v holds the leading
  left singular vectors of the upper half of the 2x2 cell ("standard").
* Sec. III and Fig. 3: the reduced environment, where the right half of that
  network is replaced by the right-move tensors {C^2, T^3} ("reduced_env" mode,
  double-layer absorption), and the further one-row approximation
  {C'^1, T'^2, C'^2}.
* Sec. IV and Fig. 4: the split isometries v = v^1 v^2 (v^1 from an SVD of the
  reduced network reshaped chi D x chi D, v^2 from an SVD of the (chi' D, chi)
  matrix) and the sequential ket-then-bra absorption.
* Appendix and Fig. 8: the auxiliary isometries v_l, v_r built from {C^1, T^1}
  and {C^2, T^3} alone.

Every SVD here is an exact LAPACK SVD (numpy.linalg.svd).  Nothing is blocked,
fused or reordered beyond the contraction sequences the paper describes.

Conventions (the figures the labels refer to carry no printed leg order, so each
of these is a reading, chosen to agree with every label the text uses):

* Site tensors A[p, u, l, d, r].  Site (i, j) holds A when i + j is even.
* Environment tensors are labelled (kind, k, x): k = 1 left, 2 top, 3 right,
  4 bottom (corners: 1 top-left, 2 top-right, 3 bottom-right, 4 bottom-left) and
  x in {'a', 'b'} the sublattice of the site they are adjacent to.  All 16
  combinations are stored (the 12 of Fig. 1d plus the corners of the window
  shifted by one site, which the reduced environment of Sec. III needs).
* Legs follow the boundary clockwise.  Corners are [prev, next]:
  C1[down, right], C2[left, down], C3[up, left], C4[right, up].  Edges are
  [prev, ket, bra, next]: T1[down, k, b, up], T2[left, k, b, right],
  T3[up, k, b, down], T4[right, k, b, left]; (k, b) attach to the site's
  outward ket and bra legs.  Fused double-layer legs put the ket index first.
* The up, right and down moves are the left move on the lattice rotated
  counter-clockwise by 1, 2, 3 quarter turns: slot k of the rotated frame holds
  slot k + r of the stored environment and the site becomes
  A.transpose(0, 4, 1, 2, 3) per quarter turn.
"""
import functools

import numpy as np

# every contraction is pairwise (two operands) and goes through BLAS-backed
# einsum; multi-operand calls are avoided because numpy's path search can pick
# outer products far larger than any tensor of the method
ein = functools.partial(np.einsum, optimize=True)

OTHER = {"a": "b", "b": "a"}
KINDS = ("C", "T")
DIRS = {"left": 0, "up": 1, "right": 2, "down": 3}
MOVE_ORDER = ("left", "up", "right", "down")


# ----------------------------------------------------------------------------
# Lattice helpers (Sec. II, Fig. 1)
# ----------------------------------------------------------------------------

def rotate_site(A, r):
    """Site tensor of the lattice rotated counter-clockwise by r quarter turns."""
    for _ in range(r % 4):
        A = A.transpose(0, 4, 1, 2, 3)
    return A


def double_layer(A):
    """Transfer tensor a = sum_p A[p,...] A*[p,...] (Fig. 1b), legs fused (ket, bra).

    Returns a[U, L, Dn, R] with each leg of dimension D^2.
    """
    D = A.shape[1]
    a = ein("puldr,pULDR->uUlLdDrR", A, A.conj())
    return a.reshape(D * D, D * D, D * D, D * D)


def slot(k, r):
    """Stored slot that plays position k in the frame rotated by r quarter turns."""
    return (k - 1 + r) % 4 + 1


class View:
    """Environment seen from the frame rotated by r quarter turns."""

    def __init__(self, env, r):
        self.env = env
        self.r = r

    def __call__(self, kind, k, x):
        return self.env[(kind, slot(k, self.r), x)]

    def put(self, kind, k, x, t):
        self.env[(kind, slot(k, self.r), x)] = t


# ----------------------------------------------------------------------------
# Initial environment by index folding
# ----------------------------------------------------------------------------

def _fold_C1(A, bnd):
    """Corner C1[down, right] of site A with its up and left legs closed by bnd."""
    D = A.shape[1]
    X = ein("puldr,uU->pUldr", A, bnd)
    X = ein("pUldr,lL->pULdr", X, bnd)
    C = ein("pULdr,pULDR->dDrR", X, A.conj())
    return C.reshape(D * D, D * D)


def _fold_T1(A, bnd):
    """Edge T1[down, k, b, up] of site A with its left leg closed by bnd."""
    D = A.shape[1]
    X = ein("puldr,lL->puLdr", A, bnd)
    T = ein("puLdr,pULDR->dDrRuU", X, A.conj())
    return T.reshape(D * D, D, D, D * D)


def fold_init(A, B, bnd=None):
    """Environment of the finite lattice whose outer legs are closed by ``bnd``.

    bnd (D x D, ket x bra) defaults to the identity, i.e. each outward ket leg is
    traced with its bra partner.  A corner C^k_x is the site diagonally outside
    x (same sublattice); an edge T^k_x is the site next to x (other sublattice).
    Bond dimensions start at chi_0 = D^2.
    """
    D = A.shape[1]
    if bnd is None:
        bnd = np.eye(D)
    site = {"a": A, "b": B}
    env = {}
    for k in range(1, 5):
        for x in "ab":
            env[("C", k, x)] = _fold_C1(rotate_site(site[x], k - 1), bnd)
            env[("T", k, x)] = _fold_T1(rotate_site(site[OTHER[x]], k - 1), bnd)
    return env


# ----------------------------------------------------------------------------
# Truncated SVD (exact)
# ----------------------------------------------------------------------------

def _sign_fix(U):
    """Make the largest-magnitude entry of every column positive."""
    idx = np.argmax(np.abs(U), axis=0)
    s = np.sign(U[idx, np.arange(U.shape[1])])
    s[s == 0] = 1.0
    return U * s


def trunc_left(Mmat, k):
    """Leading k left singular vectors of Mmat (rows x cols).

    When k reaches the row count the bond is not truncated and the identity is
    returned (any orthonormal basis of the full space is gauge-equivalent).
    """
    m = Mmat.shape[0]
    if k >= m:
        return np.eye(m)
    U, s, _ = np.linalg.svd(Mmat, full_matrices=False)
    if U.shape[1] < k:
        raise ValueError("truncation rank exceeds the matrix rank bound")
    return _sign_fix(U[:, :k])


# ----------------------------------------------------------------------------
# Absorption primitives
# ----------------------------------------------------------------------------

def edge_site_T1(A):
    """Site legs in edge-local order (p, in, out, prev, next) for a left-edge absorption."""
    return A.transpose(0, 2, 4, 3, 1)


def edge_site_T2(A):
    """Site legs in edge-local order (p, in, out, prev, next) for a top-edge absorption."""
    return A.transpose(0, 1, 3, 2, 4)


def absorb_edge_double(T, S, vp, vn):
    """Double-layer edge absorption with 4-index projectors (Sec. II, Fig. 2b).

    T[prev, k, b, next], S[p, in, out, prev_leg, next_leg],
    vp[prev, pk, pb, chi_p], vn[next, nk, nb, chi_n].
    Returns T_new[chi_p, out_k, out_b, chi_n].
    """
    a = ein("pioqn,pIOQN->iIoOqQnN", S, S.conj())
    X = ein("AkbB,kbOPqQnN->AOPqQBnN", T, a)
    X = ein("AOPqQBnN,AqQx->xOPBnN", X, vp)
    return ein("xOPBnN,BnNy->xOPy", X, vn)


def absorb_edge_seq(T, S, vp1, vp2, vn1, vn2):
    """Sequential (ket, then bra) edge absorption with split projectors (Sec. IV, Fig. 4b).

    v^1 contracts the boundary leg of T with the ket leg of the site; v^2
    contracts the intermediate leg of v^1 with the bra leg.  Six pairwise
    contractions, each O(chi^3 D^3) at chi' = chi.
    T[prev, k, b, next], S[p, in, out, prev_leg, next_leg],
    vp1[prev, pk, c_p], vp2[c_p, pb, chi_p], vn1[next, nk, c_n], vn2[c_n, nb, chi_n].
    """
    X1 = ein("AkbB,Bnc->Akbnc", T, vn1)                 # over the next boundary leg
    X2 = ein("Akbnc,skoqn->Abcsoq", X1, S)               # ket site over (in, next)
    X3 = ein("Abcsoq,Aqe->bcsoe", X2, vp1)               # over (prev boundary, prev ket)
    X4 = ein("bcsoe,cNy->bsoeNy", X3, vn2)               # over the next intermediate leg
    X5 = ein("bsoeNy,sbOQN->oeyOQ", X4, S.conj())        # bra site over (p, in, next)
    return ein("oeyOQ,eQx->xoOy", X5, vp2)               # over (prev intermediate, prev bra)


def compose(v1, v2):
    """4-index isometry v[chi, k, b, chi_new] = sum_c v1[chi, k, c] v2[c, b, chi_new]."""
    return ein("akc,cby->akby", v1, v2)


def corner_C1_absorb(C1, T2, v):
    """New C1[down, right] = v^T (C1 T2) on the down bond (Fig. 2a, b)."""
    X = ein("dg,gkbe->dkbe", C1, T2)
    return ein("dkbe,dkby->ye", X, v)


def corner_C4_absorb(C4, T4, v):
    """New C4[right, up] = (C4 T4) v on the up bond (Fig. 2a, b)."""
    X = ein("lu,rkbl->rukb", C4, T4)
    return ein("rukb,ukby->ry", X, v)


# ----------------------------------------------------------------------------
# Projectors
# ----------------------------------------------------------------------------

def projector_standard(V, x, sites, chi):
    """v_{x/y} for the bond below x from the 8-tensor upper half (Sec. II, Fig. 2c).

    Q[(alpha, Dx), (Dy, beta)] = E_L E_R with
    E_L = {C1_x, T2_x, T1_x, a_x} and E_R = {T2_y, C2_y, a_y, T3_y};
    v = leading min(chi, rows) left singular vectors, reshaped (alpha, D, D, chi).
    """
    y = OTHER[x]
    D = sites[x].shape[1]
    ax, ay = double_layer(sites[x]), double_layer(sites[y])
    C1, T1 = V("C", 1, x), V("T", 1, x)
    T2x, T2y = V("T", 2, x), V("T", 2, y)
    C2, T3 = V("C", 2, y), V("T", 3, y)
    T1f = T1.reshape(T1.shape[0], D * D, T1.shape[3])
    T2xf = T2x.reshape(T2x.shape[0], D * D, T2x.shape[3])
    T2yf = T2y.reshape(T2y.shape[0], D * D, T2y.shape[3])
    T3f = T3.reshape(T3.shape[0], D * D, T3.shape[3])
    EL = ein("dg,gUe->dUe", C1, T2xf)
    EL = ein("dUe,aLd->aLUe", EL, T1f)
    EL = ein("aLUe,ULXR->aXeR", EL, ax)
    ER = ein("eUz,zh->eUh", T2yf, C2)
    ER = ein("eUh,hRb->eURb", ER, T3f)
    ER = ein("eURb,ULYR->eLbY", ER, ay)
    Q = ein("aXeR,eRbY->aXYb", EL, ER)
    na = Q.shape[0]
    Qm = Q.reshape(na * D * D, -1)
    v = trunc_left(Qm, min(chi, na * D * D))
    return v.reshape(na, D, D, v.shape[1])


def projector_reduced_env(V, x, sites, chi):
    """v_{x/y} for the bond below x from the reduced environment (Sec. III, Fig. 3a-b).

    The right half {y, T2_y, C2_y, T3_y} of the standard upper half is replaced
    by the right-move tensors {C2_x, T3_x}; the isometry v of that right move
    is dropped, leaving Q = E_L (C2_x T3_x), a (chi D^2) x chi matrix whose
    leading min(chi, rows) left singular vectors give v (alpha, D, D, chi).
    """
    D = sites[x].shape[1]
    ax = double_layer(sites[x])
    C1, T1, T2x = V("C", 1, x), V("T", 1, x), V("T", 2, x)
    C2, T3 = V("C", 2, x), V("T", 3, x)
    T1f = T1.reshape(T1.shape[0], D * D, T1.shape[3])
    T2xf = T2x.reshape(T2x.shape[0], D * D, T2x.shape[3])
    T3f = T3.reshape(T3.shape[0], D * D, T3.shape[3])
    EL = ein("dg,gUe->dUe", C1, T2xf)
    EL = ein("dUe,aLd->aLUe", EL, T1f)
    EL = ein("aLUe,ULXR->aXeR", EL, ax)
    R = ein("ez,zRb->eRb", C2, T3f)
    Q = ein("aXeR,eRb->aXb", EL, R)
    na, nb = Q.shape[0], Q.shape[2]
    v = trunc_left(Q.reshape(na * D * D, nb), min(chi, na * D * D))
    return v.reshape(na, D, D, v.shape[1])


def split_projector(Mt, chi, chip):
    """Split isometries from a 4-leg network Mt[alpha, k, b, beta] (Sec. IV, Fig. 4a).

    v1 = leading min(chi', alpha*D) left singular vectors of Mt reshaped
    (alpha k) x (b beta); then N = v1^T Mt reshaped (c b) x beta gives
    v2 = leading min(chi, c*D) left singular vectors.
    """
    na, D, _, nb = Mt.shape
    v1 = trunc_left(Mt.reshape(na * D, D * nb), min(chip, na * D))
    k1 = v1.shape[1]
    v1 = v1.reshape(na, D, k1)
    N = ein("akc,akbz->cbz", v1, Mt)
    v2 = trunc_left(N.reshape(k1 * D, nb), min(chi, k1 * D))
    v2 = v2.reshape(k1, D, v2.shape[1])
    return v1, v2


def reduced_network(V, x, sites, chi, chip):
    """The one-row reduced network M = C'1 T'2 C'2 for the bond below x (Fig. 3c, Fig. 8).

    v_l comes from L = C1_x T1_x and v_r from R = C2_x T3_x (Appendix); C'1 and
    C'2 are L and R projected on their horizontal bond and T'2 is T2_x with the
    site x absorbed sequentially.  Returns M[alpha, d_k, d_b, beta].
    """
    C1, T1 = V("C", 1, x), V("T", 1, x)
    C2, T3 = V("C", 2, x), V("T", 3, x)
    T2 = V("T", 2, x)
    L = ein("dg,akbd->gkba", C1, T1)       # [C1.right, k, b, T1.down]
    R = ein("ez,zkbw->ekbw", C2, T3)       # [C2.left, k, b, T3.down]
    vl1, vl2 = split_projector(L, chi, chip)
    vr1, vr2 = split_projector(R, chi, chip)
    C1p = ein("cby,cba->ya", vl2, ein("gkc,gkba->cba", vl1, L))
    C2p = ein("cby,cbw->yw", vr2, ein("ekc,ekbw->cbw", vr1, R))
    T2p = absorb_edge_seq(T2, edge_site_T2(sites[x]), vl1, vl2, vr1, vr2)
    return ein("akbz,zw->akbw", ein("ya,ykbz->akbz", C1p, T2p), C2p)


def projector_reduced_seq(V, x, sites, chi, chip):
    """(v1, v2) for the bond below x from the reduced network (Sec. IV, Appendix)."""
    return split_projector(reduced_network(V, x, sites, chi, chip), chi, chip)


# ----------------------------------------------------------------------------
# Moves
# ----------------------------------------------------------------------------

def _normalize(t):
    n = np.linalg.norm(t)
    if not np.isfinite(n) or n == 0.0:
        raise FloatingPointError("environment tensor norm is zero or not finite")
    return t / n


def column_absorb(env, r, sites_r, chi, chip, mode):
    """Absorb one column into the boundary of frame r (Sec. II, Fig. 2a).

    Every left-boundary tensor adjacent to x becomes the one adjacent to the
    other sublattice: C1_x T2_x -> C1_y, T1_x x -> T1_y, C4_x T4_x -> C4_y.  The
    bond below x is truncated by P_{x/y} and the bond above x by P_{y/x}.
    """
    V = View(env, r)
    P = {}
    for x in "ab":
        if mode == "standard":
            P[x] = projector_standard(V, x, sites_r, chi)
        elif mode == "reduced_env":
            P[x] = projector_reduced_env(V, x, sites_r, chi)
        elif mode == "reduced_sequential":
            P[x] = projector_reduced_seq(V, x, sites_r, chi, chip)
        else:
            raise ValueError(mode)
    new = {}
    for x in "ab":
        y = OTHER[x]
        S = edge_site_T1(sites_r[x])
        if mode in ("standard", "reduced_env"):
            vb, vt = P[x], P[y]
            new[("T", 1, y)] = absorb_edge_double(V("T", 1, x), S, vb, vt)
        else:
            (b1, b2), (t1, t2) = P[x], P[y]
            new[("T", 1, y)] = absorb_edge_seq(V("T", 1, x), S, b1, b2, t1, t2)
            vb, vt = compose(b1, b2), compose(t1, t2)
        new[("C", 1, y)] = corner_C1_absorb(V("C", 1, x), V("T", 2, x), vt)
        new[("C", 4, y)] = corner_C4_absorb(V("C", 4, x), V("T", 4, x), vb)
    for (kind, k, x), t in new.items():
        V.put(kind, k, x, _normalize(t))
    return P


def move(env, direction, A, B, chi, chip=None, mode="reduced_sequential"):
    """One CTM move (two column absorptions, Sec. II) in direction left/up/right/down."""
    r = DIRS[direction]
    chip = chi if chip is None else chip
    sites_r = {"a": rotate_site(A, r), "b": rotate_site(B, r)}
    column_absorb(env, r, sites_r, chi, chip, mode)
    column_absorb(env, r, sites_r, chi, chip, mode)
    return env


def bond_dims(env):
    return {key: t.shape for key, t in env.items()}


def grow(env, A, B, chi, max_iter=16):
    """Grow the folded environment to bond dimension chi with standard moves.

    The reduced networks of Sec. III and IV have rank at most the bond
    dimension of the right-move tensors, so they cannot grow a bond; the
    standard move does, and is used until no bond changes.
    """
    for _ in range(max_iter):
        before = bond_dims(env)
        if all(min(s[0], s[-1]) >= chi for s in before.values()):
            break
        for d in MOVE_ORDER:
            move(env, d, A, B, chi, chi, "standard")
        if bond_dims(env) == before:
            break
    return env


def init_env(A, B, chi, bnd=None):
    """Folded environment grown to bond dimension chi (ctm_init_env)."""
    env = fold_init(A, B, bnd)
    env = {key: _normalize(t) for key, t in env.items()}
    return grow(env, A, B, chi)


# ----------------------------------------------------------------------------
# Gauge-invariant outputs
# ----------------------------------------------------------------------------

CORNER_ORDER = [(k, x) for k in range(1, 5) for x in "ab"]


def corner_spectra(env):
    """Singular values of the 8 corners (C1a, C1b, ..., C4b), each scaled to sum s^2 = 1."""
    out = []
    for k, x in CORNER_ORDER:
        s = np.linalg.svd(env[("C", k, x)], compute_uv=False)
        out.append(s / np.linalg.norm(s))
    return out


def spectrum_delta(old, new):
    d = 0.0
    for s0, s1 in zip(old, new):
        n = max(len(s0), len(s1))
        a = np.zeros(n); a[: len(s0)] = s0
        b = np.zeros(n); b[: len(s1)] = s1
        d = max(d, float(np.linalg.norm(a - b)))
    return d


def converge(env, A, B, chi, chip=None, mode="reduced_sequential", max_iter=50, tol=1e-10):
    """Iterate left, up, right, down moves until the corner spectra change by < tol."""
    spec = corner_spectra(env)
    delta = np.inf
    it = 0
    for it in range(1, max_iter + 1):
        for d in MOVE_ORDER:
            move(env, d, A, B, chi, chip, mode)
        new = corner_spectra(env)
        delta = spectrum_delta(spec, new)
        spec = new
        if delta < tol:
            break
    return it, delta


def _open_double(A):
    """a[p, p', U, L, Dn, R] with the physical legs left open."""
    D, d = A.shape[1], A.shape[0]
    a = ein("puldr,PULDR->pPuUlLdDrR", A, A.conj())
    return a.reshape(d, d, D * D, D * D, D * D, D * D)


def bond_rdm(env, A, B, r, x):
    """Two-site density matrix rho[(i j), (i' j')] of the horizontal pair (x, y) in frame r."""
    y = OTHER[x]
    V = View(env, r)
    site = {"a": rotate_site(A, r), "b": rotate_site(B, r)}
    D, d = A.shape[1], A.shape[0]
    f = lambda t: t.reshape(t.shape[0], D * D, t.shape[3])
    C1, T2x, T2y, C2 = V("C", 1, x), f(V("T", 2, x)), f(V("T", 2, y)), V("C", 2, y)
    T3, C3, T4y, T4x = f(V("T", 3, y)), V("C", 3, y), f(V("T", 4, y)), f(V("T", 4, x))
    C4, T1 = V("C", 4, x), f(V("T", 1, x))
    ax, ay = _open_double(site[x]), _open_double(site[y])
    left = ein("dg,gUe->dUe", C1, T2x)
    left = ein("dUe,mLd->mLUe", left, T1)
    left = ein("mLUe,lm->lLUe", left, C4)
    left = ein("lLUe,kXl->kXLUe", left, T4x)
    left = ein("kXLUe,pPULXR->eRkpP", left, ax)
    right = ein("eVz,zh->eVh", T2y, C2)
    right = ein("eVh,hWt->eVWt", right, T3)
    right = ein("eVWt,ti->eVWi", right, C3)
    right = ein("eVWi,iYk->eVWYk", right, T4y)
    right = ein("eVWYk,qQVRYW->eRkqQ", right, ay)
    rho = ein("eRkpP,eRkqQ->pqPQ", left, right)
    return rho.reshape(d * d, d * d)


BONDS = {0: (0, "a"), 1: (0, "b"), 2: (1, "a"), 3: (1, "b")}


def bond_rdm_seq(env, A, B, r, x):
    """The same density matrix as ``bond_rdm``, with each site's ket layer and bra
    layer absorbed one after the other (the order of Sec. IV applied to the
    observable) instead of through the open double-layer tensor: the largest
    intermediate is chi^2 d^2 D^4 instead of chi^2 D^6, which makes the energy
    computable at D = 6..8."""
    y = OTHER[x]
    V = View(env, r)
    Sx, Sy = rotate_site({"a": A, "b": B}[x], r), rotate_site({"a": A, "b": B}[y], r)
    d = A.shape[0]
    # left half: frame (C1 T2 T1) with the ket and bra of x, closed by (T4 C4)
    top = ein("dg,gKBe->dKBe", V("C", 1, x), V("T", 2, x))        # [down, Uk, Ub, e]
    top = ein("dKBe,mLld->mLlKBe", top, V("T", 1, x))              # [m, Lk, Lb, Uk, Ub, e]
    ket = ein("mLlKBe,pKLnr->mlBepnr", top, Sx)                     # ket: u = Uk, l = Lk
    both = ein("mlBepnr,PBlNR->mepnrPNR", ket, Sx.conj())           # bra: u = Ub, l = Lb
    bot = ein("jnNo,om->jnNm", V("T", 4, x), V("C", 4, x))          # T4 [right, k, b, left]
    left = ein("mepnrPNR,jnNm->ejrRpP", both, bot)                  # [e, j, Rk, Rb, p, P]
    # right half: frame (T2 C2 T3) with the ket and bra of y, closed by (C3 T4)
    top = ein("eKBz,zh->eKBh", V("T", 2, y), V("C", 2, y))          # [e, Uk, Ub, h]
    top = ein("eKBh,hWwt->eKBWwt", top, V("T", 3, y))               # [e, Uk, Ub, Rk, Rb, t]
    ket = ein("eKBWwt,qKlnW->eBwtqln", top, Sy)                     # ket: u = Uk, r = Rk
    both = ein("eBwtqln,QBLNw->etqlnQLN", ket, Sy.conj())           # bra: u = Ub, r = Rb
    bot = ein("ti,inNj->tnNj", V("C", 3, y), V("T", 4, y))          # T4 [right, k, b, left]
    right = ein("etqlnQLN,tnNj->ejlLqQ", both, bot)                 # [e, j, Lk, Lb, q, Q]
    rho = ein("ejrRpP,ejrRqQ->pqPQ", left, right)
    return rho.reshape(d * d, d * d)


def expect_bond_seq(env, A, B, bond, op):
    """``expect_bond`` through ``bond_rdm_seq`` (for D where the open double layer
    does not fit)."""
    r, x = BONDS[bond]
    rho = bond_rdm_seq(env, A, B, r, x)
    return float(np.trace(rho @ op) / np.trace(rho))



def expect_bond(env, A, B, bond, op):
    """<op> on a nearest-neighbour bond: 0 = a-b horizontal, 1 = b-a horizontal,
    2 = a above b, 3 = b above a.  op is (d^2 x d^2) with rows/cols (i_x, i_y)."""
    r, x = BONDS[bond]
    rho = bond_rdm(env, A, B, r, x)
    return float(np.trace(rho @ op) / np.trace(rho))


def heisenberg_bond():
    """h = S_i . S_j with S = sigma / 2 (real: Sy Sy is real)."""
    sx = np.array([[0, 1], [1, 0]], float) / 2
    sz = np.array([[1, 0], [0, -1]], float) / 2
    sy_sy = -np.kron(np.array([[0, -1], [1, 0]], float), np.array([[0, -1], [1, 0]], float)) / 4
    return np.kron(sx, sx) + sy_sy + np.kron(sz, sz)


def _trace_net(tensors, spec):
    """Close a ring of tensors pairwise, left to right, in the order given."""
    ins, _ = spec.split("->")
    labels = ins.split(",")
    acc, acc_l = tensors[0], labels[0]
    for t, lab in zip(tensors[1:], labels[1:]):
        keep = [ch for ch in acc_l + lab if (acc_l + lab).count(ch) == 1]
        out = "".join(keep)
        acc = ein(f"{acc_l},{lab}->{out}", acc, t)
        acc_l = out
    return float(acc)


def _log_kappa_from(V, x, y):
    """Z00, Z20, Z02 of the window with top-left sublattice x (corner labels follow
    the site each corner touches: C1 at (i, j), C2 at (i, j+w-1), C3 at
    (i+h-1, j+w-1), C4 at (i+h-1, j) for an h x w block)."""
    D2 = V("T", 1, x).shape[1] * V("T", 1, x).shape[2]
    f = lambda t: t.reshape(t.shape[0], D2, t.shape[3])
    # Z00: corners around an empty window
    z00 = _trace_net([V("C", 1, x), V("C", 2, y), V("C", 3, x), V("C", 4, y)],
                     "ab,bc,cd,da->")
    # Z20: two rows, no columns
    z20 = _trace_net([V("C", 1, x), V("C", 2, y), f(V("T", 3, y)), f(V("T", 3, x)),
                      V("C", 3, x), V("C", 4, y), f(V("T", 1, y)), f(V("T", 1, x))],
                     "ab,bc,cKd,dLe,ef,fg,gLh,hKa->")
    # Z02: no rows, two columns
    z02 = _trace_net([V("C", 1, x), f(V("T", 2, x)), f(V("T", 2, y)), V("C", 2, y),
                      V("C", 3, x), f(V("T", 4, x)), f(V("T", 4, y)), V("C", 4, y)],
                     "ab,bKc,cLd,de,ef,fLg,gKh,ha->")
    return z00, z20, z02


def log_kappa_sites(env, A, B, x="a"):
    """ln kappa per site from the 2x2 window with top-left site x."""
    y = OTHER[x]
    V = View(env, 0)
    site = {"a": A, "b": B}
    D = A.shape[1]
    f = lambda t: t.reshape(t.shape[0], D * D, t.shape[3])
    z00, z20, z02 = _log_kappa_from(V, x, y)
    ax, ay = double_layer(site[x]), double_layer(site[y])
    # Z22: the whole window, contracted as an upper and a lower row
    E = ein("dg,gPc->dPc", V("C", 1, x), f(V("T", 2, x)))
    E = ein("dPc,lWd->lWPc", E, f(V("T", 1, x)))
    E = ein("lWPc,PWXY->lcXY", E, ax)
    F = ein("cQe,eh->cQh", f(V("T", 2, y)), V("C", 2, y))
    F = ein("cQh,hRf->cQRf", F, f(V("T", 3, y)))
    F = ein("cQRf,QYZR->cfYZ", F, ay)
    up = ein("lcXY,cfYZ->lXfZ", E, F)
    G = ein("jk,kVl->jVl", V("C", 4, y), f(V("T", 1, y)))
    G = ein("jVl,iUj->iUVl", G, f(V("T", 4, y)))
    G = ein("iUVl,XVUN->ilXN", G, ay)
    H = ein("gh,hTi->gTi", V("C", 3, x), f(V("T", 4, x)))
    H = ein("gTi,fSg->fSTi", H, f(V("T", 3, x)))
    H = ein("fSTi,ZNTS->fiZN", H, ax)
    low = ein("ilXN,fiZN->lXfZ", G, H)
    z22 = float(ein("lXfZ,lXfZ->", up, low))
    ratio = z22 * z00 / (z20 * z02)
    if not ratio > 0:
        raise FloatingPointError("non-positive norm ratio")
    return 0.25 * float(np.log(ratio))


# ----------------------------------------------------------------------------
# Row transfer: correlation function along a row (Sec. V, Fig. 9b)
# ----------------------------------------------------------------------------

def _strip_absorb(V, T2, S, op, T4):
    """Absorb one column (T2 above, site S with `op` between ket and bra
    physical legs, T4 below) into the strip vector V[top, k, b, bottom]."""
    W = ein("tkbr,tKBu->kbrKBu", V, T2)
    W = ein("kbrKBu,pKkDq->brBupDq", W, S)          # ket: (p, up, left, down, right)
    W = ein("brBupDq,Pp->brBuPDq", W, op)            # <psi| op |psi>: op[bra, ket]
    W = ein("brBuPDq,PBbEQ->ruDqEQ", W, S.conj())    # bra
    return ein("ruDqEQ,vDEr->uqQv", W, T4)


def _strip_close(V, C2, T3, C3):
    X = ein("uqQv,ue->eqQv", V, C2)
    X = ein("eqQv,eqQg->gv", X, T3)
    return float(ein("gv,gv->", X, C3))


def row_correlator(env, A, B, op1, op2, xmax):
    """S(x) = <op1_0 op2_x> - <op1_0><op2_x> for sites 0..x of a row starting on
    sublattice a, x = 1..xmax, from the strip closed by C1_a T1_a C4_a on the left
    and by C2, T3, C3 of the last site on the right (Sec. V: S_zz(x))."""
    site = {"a": A, "b": B}
    d = A.shape[0]
    ident = np.eye(d)
    V0 = ein("dt,akbd->tkba", env[("C", 1, "a")], env[("T", 1, "a")])
    V0 = ein("tkba,ra->tkbr", V0, env[("C", 4, "a")])
    T2, T4 = env[("T", 2, "a")], env[("T", 4, "a")]
    Vid = _strip_absorb(V0, T2, A, ident, T4)
    Vop = _strip_absorb(V0, T2, A, op1, T4)
    out = []
    for x in range(1, xmax + 1):
        s = "a" if x % 2 == 0 else "b"
        T2, T4, S = env[("T", 2, s)], env[("T", 4, s)], site[s]
        C2, T3, C3 = env[("C", 2, s)], env[("T", 3, s)], env[("C", 3, s)]
        nid = _strip_absorb(Vid, T2, S, ident, T4)
        nop = _strip_absorb(Vop, T2, S, ident, T4)
        z = _strip_close(nid, C2, T3, C3)
        one0 = _strip_close(nop, C2, T3, C3) / z
        onex = _strip_close(_strip_absorb(Vid, T2, S, op2, T4), C2, T3, C3) / z
        two = _strip_close(_strip_absorb(Vop, T2, S, op2, T4), C2, T3, C3) / z
        out.append(two - one0 * onex)
        scale = np.linalg.norm(nid)
        Vid, Vop = nid / scale, nop / scale
    return np.array(out)
