"""Reverse-mode derivative of the CTM bond energy with respect to the site tensors
(plain PyTorch on the CPU, FP64).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or calls
this module; only ``tests/`` may use it.  It shares no code with the CUDA path.

What it computes: the Heisenberg energy per bond (mean of the four bonds of the
2-site cell, Eq. 1 with S = sigma/2) after ``iters`` CTM iterations of the
reduced-sequential move (Sec. III, IV, Appendix) started from a given
environment, and its gradient with respect to A and B.  The starting environment
is held fixed (a constant of the loss); the gradient runs back through every
sequential absorption (Fig. 4b), every projector application and every truncated
SVD of the projectors (Fig. 4a, Fig. 8).

The forward steps are those of ``oracle.ctm_oracle`` written with torch tensor
operations (pairwise einsums, LAPACK SVD), so that torch.autograd differentiates
them.  The one hand-written adjoint is the truncated SVD's (``TruncatedLeft``):
for A = U S V^T (thin), with only the leading k columns of U used,

    dA = U [ (F o (U^T dU - dU^T U)) S ] V^T + (I - U U^T) dU S^-1 V^T

where dU is the incoming gradient zero-padded to all columns and
F_ij = 1 / (s_j^2 - s_i^2) off the diagonal, broadened to
(s_j^2 - s_i^2) / ((s_j^2 - s_i^2)^2 + eps s_max^4) (Liao, Liu, Wang & Xiang,
PRX 9, 031041 (2019), there with s_max = 1) so that degenerate pairs contribute
zero instead of dividing by zero; with eps = 0 an exactly degenerate pair is
given F_ij = 0 and a zero singular value the pseudo-inverse 0 in S^-1 (the
eps -> 0+ limits of the broadened forms).  The broadening is relative to the largest
singular value: the matrices of a CTM move carry no fixed scale.  The second
term carries the part of dU outside the span of U (Townsend, "Differentiating
the singular value decomposition", 2016).  S and V^T receive no
gradient here because a projector v v^T uses the left vectors only.
"""
import torch
import torch.utils.checkpoint

from oracle import ctm_oracle as O

DT = torch.float64


def ein(spec, a, b):
    return torch.einsum(spec, a, b)


# ----------------------------------------------------------------------------
# Truncated SVD with a broadened adjoint
# ----------------------------------------------------------------------------

class TruncatedLeft(torch.autograd.Function):
    """Leading k left singular vectors of M (rows x cols), largest-magnitude entry
    of each column made positive (the oracle's sign convention)."""

    @staticmethod
    def forward(ctx, M, k, eps):
        U, S, Vh = torch.linalg.svd(M, full_matrices=False)
        if U.shape[1] < k:
            raise ValueError("truncation rank exceeds the matrix rank bound")
        Uk = U[:, :k]
        idx = torch.argmax(Uk.abs(), dim=0)
        sign = torch.sign(Uk[idx, torch.arange(k)])
        sign[sign == 0] = 1.0
        ctx.save_for_backward(U, S, Vh, sign)
        ctx.k, ctx.eps = k, eps
        return Uk * sign

    @staticmethod
    def backward(ctx, g):
        U, S, Vh, sign = ctx.saved_tensors
        return svd_left_adjoint(U, S, Vh, g * sign, ctx.eps), None, None


def svd_left_adjoint(U, S, Vh, gUk, eps):
    """dM for M = U diag(S) Vh (thin, S descending) given the gradient gUk of the
    leading k = gUk.shape[1] columns of U (the formula of the module docstring)."""
    m, r = U.shape
    k = gUk.shape[1]
    gU = torch.zeros_like(U)
    gU[:, :k] = gUk
    J = U.T @ gU
    E = S[None, :] ** 2 - S[:, None] ** 2          # E_ij = s_j^2 - s_i^2
    den = E * E + eps * S[0] ** 4                    # eps relative to s_max^4
    # a pair with den = 0 (exactly degenerate, no broadening) contributes zero:
    # the eps -> 0+ limit of the broadened factor at E = 0
    F = torch.where(den > 0, E / torch.where(den > 0, den, torch.ones_like(den)),
                    torch.zeros_like(E))
    F.fill_diagonal_(0.0)
    inner = (F * (J - J.T)) * S[None, :]             # (F o skew) S
    gM = U @ inner @ Vh
    if m > r:  # part of dU outside span(U); only the kept columns are non-zero
        gperp = gU - U @ J
        # pseudo-inverse of S: a zero singular value contributes zero (the limit
        # of the broadened inverse s / (s^2 + eps) at s = 0)
        sk = S[:k]
        inv = torch.where(sk > 0, 1.0 / torch.where(sk > 0, sk, torch.ones_like(sk)),
                          torch.zeros_like(sk))
        gM = gM + (gperp[:, :k] * inv[None, :]) @ Vh[:k, :]
    return gM


def trunc_left(M, k, eps):
    """Leading k left singular vectors; the identity (a constant) when k reaches the rows."""
    m = M.shape[0]
    if k >= m:
        return torch.eye(m, dtype=DT)
    return TruncatedLeft.apply(M, k, eps)


# ----------------------------------------------------------------------------
# Reduced-sequential move (same steps as oracle.ctm_oracle)
# ----------------------------------------------------------------------------

def rotate_site(A, r):
    for _ in range(r % 4):
        A = A.permute(0, 4, 1, 2, 3)
    return A


def edge_site_T1(A):
    return A.permute(0, 2, 4, 3, 1)


def edge_site_T2(A):
    return A.permute(0, 1, 3, 2, 4)


def absorb_edge_seq(T, S, vp1, vp2, vn1, vn2):
    """Sec. IV, Fig. 4b: ket site, then bra site, six pairwise contractions."""
    X1 = ein("AkbB,Bnc->Akbnc", T, vn1)
    X2 = ein("Akbnc,skoqn->Abcsoq", X1, S)
    X3 = ein("Abcsoq,Aqe->bcsoe", X2, vp1)
    X4 = ein("bcsoe,cNy->bsoeNy", X3, vn2)
    X5 = ein("bsoeNy,sbOQN->oeyOQ", X4, S)
    return ein("oeyOQ,eQx->xoOy", X5, vp2)


def contract_adjoint(spec, A, B, gC):
    """(dA, dB) for C = einsum(spec, A, B) given dC: each is one more pairwise
    contraction, of dC with the other operand (every index of A and B appears in
    exactly two of A, B, C, as in every contraction of the move)."""
    ins, out = spec.split("->")
    a, b = ins.split(",")
    return ein(f"{out},{b}->{a}", gC, B), ein(f"{a},{out}->{b}", A, gC)


ABSORB_SEQ_SPECS = ("AkbB,Bnc->Akbnc", "Akbnc,skoqn->Abcsoq", "Abcsoq,Aqe->bcsoe",
                    "bcsoe,cNy->bsoeNy", "bsoeNy,sbOQN->oeyOQ", "oeyOQ,eQx->xoOy")


def absorb_edge_seq_adjoint(T, S, vp1, vp2, vn1, vn2, gOut):
    """Hand-written reverse pass of absorb_edge_seq (Sec. IV, Fig. 4b): the six
    contractions recomputed, then walked backwards with contract_adjoint.  Returns
    (dT, dS, dvp1, dvp2, dvn1, dvn2); S enters twice (ket and bra), so dS is the sum
    of both uses."""
    sp = ABSORB_SEQ_SPECS
    X1 = ein(sp[0], T, vn1)
    X2 = ein(sp[1], X1, S)
    X3 = ein(sp[2], X2, vp1)
    X4 = ein(sp[3], X3, vn2)
    X5 = ein(sp[4], X4, S)
    gX5, gvp2 = contract_adjoint(sp[5], X5, vp2, gOut)
    gX4, gS_bra = contract_adjoint(sp[4], X4, S, gX5)
    gX3, gvn2 = contract_adjoint(sp[3], X3, vn2, gX4)
    gX2, gvp1 = contract_adjoint(sp[2], X2, vp1, gX3)
    gX1, gS_ket = contract_adjoint(sp[1], X1, S, gX2)
    gT, gvn1 = contract_adjoint(sp[0], T, vn1, gX1)
    return gT, gS_ket + gS_bra, gvp1, gvp2, gvn1, gvn2


def compose(v1, v2):
    return ein("akc,cby->akby", v1, v2)


def corner_C1_absorb(C1, T2, v):
    return ein("dkbe,dkby->ye", ein("dg,gkbe->dkbe", C1, T2), v)


def corner_C4_absorb(C4, T4, v):
    return ein("rukb,ukby->ry", ein("lu,rkbl->rukb", C4, T4), v)


def split_projector(Mt, chi, chip, eps):
    """Sec. IV, Fig. 4a: v1 from Mt as (alpha k) x (b beta), v2 from v1^T Mt as (c b) x beta."""
    na, D, _, nb = Mt.shape
    v1 = trunc_left(Mt.reshape(na * D, D * nb), min(chip, na * D), eps)
    k1 = v1.shape[1]
    v1 = v1.reshape(na, D, k1)
    N = ein("akc,akbz->cbz", v1, Mt)
    v2 = trunc_left(N.reshape(k1 * D, nb), min(chi, k1 * D), eps)
    return v1, v2.reshape(k1, D, v2.shape[1])


def reduced_network(V, x, sites, chi, chip, eps):
    """Fig. 3c, Fig. 8: M = C'1 T'2 C'2 with v_l from C1 T1 and v_r from C2 T3."""
    C1, T1 = V("C", 1, x), V("T", 1, x)
    C2, T3 = V("C", 2, x), V("T", 3, x)
    T2 = V("T", 2, x)
    L = ein("dg,akbd->gkba", C1, T1)
    R = ein("ez,zkbw->ekbw", C2, T3)
    vl1, vl2 = split_projector(L, chi, chip, eps)
    vr1, vr2 = split_projector(R, chi, chip, eps)
    C1p = ein("cby,cba->ya", vl2, ein("gkc,gkba->cba", vl1, L))
    C2p = ein("cby,cbw->yw", vr2, ein("ekc,ekbw->cbw", vr1, R))
    T2p = absorb_edge_seq(T2, edge_site_T2(sites[x]), vl1, vl2, vr1, vr2)
    return ein("akbz,zw->akbw", ein("ya,ykbz->akbz", C1p, T2p), C2p)


def column_absorb(env, r, sites_r, chi, chip, eps):
    """Sec. II, Fig. 2a with the reduced-sequential projectors of Sec. IV."""
    V = O.View(env, r)
    P = {x: split_projector(reduced_network(V, x, sites_r, chi, chip, eps), chi, chip, eps)
         for x in "ab"}
    new = {}
    for x in "ab":
        y = O.OTHER[x]
        (b1, b2), (t1, t2) = P[x], P[y]
        new[("T", 1, y)] = absorb_edge_seq(V("T", 1, x), edge_site_T1(sites_r[x]), b1, b2, t1, t2)
        new[("C", 1, y)] = corner_C1_absorb(V("C", 1, x), V("T", 2, x), compose(t1, t2))
        new[("C", 4, y)] = corner_C4_absorb(V("C", 4, x), V("T", 4, x), compose(b1, b2))
    for (kind, k, x), t in new.items():
        V.put(kind, k, x, t / torch.linalg.norm(t))


def move(env, direction, A, B, chi, chip, eps):
    r = O.DIRS[direction]
    sites_r = {"a": rotate_site(A, r), "b": rotate_site(B, r)}
    column_absorb(env, r, sites_r, chi, chip, eps)
    column_absorb(env, r, sites_r, chi, chip, eps)


# ----------------------------------------------------------------------------
# Energy
# ----------------------------------------------------------------------------

def bond_rdm(env, A, B, r, x):
    """Two-site density matrix of the horizontal pair (x, y) in frame r (as the oracle's)."""
    y = O.OTHER[x]
    V = O.View(env, r)
    site = {"a": rotate_site(A, r), "b": rotate_site(B, r)}
    d, D = A.shape[0], A.shape[1]
    f = lambda t: t.reshape(t.shape[0], D * D, t.shape[3])
    dbl = lambda S: ein("puldr,PULDR->pPuUlLdDrR", S, S).reshape(d, d, D * D, D * D, D * D, D * D)
    left = ein("dg,gUe->dUe", V("C", 1, x), f(V("T", 2, x)))
    left = ein("dUe,mLd->mLUe", left, f(V("T", 1, x)))
    left = ein("mLUe,lm->lLUe", left, V("C", 4, x))
    left = ein("lLUe,kXl->kXLUe", left, f(V("T", 4, x)))
    left = ein("kXLUe,pPULXR->eRkpP", left, dbl(site[x]))
    right = ein("eVz,zh->eVh", f(V("T", 2, y)), V("C", 2, y))
    right = ein("eVh,hWt->eVWt", right, f(V("T", 3, y)))
    right = ein("eVWt,ti->eVWi", right, V("C", 3, y))
    right = ein("eVWi,iYk->eVWYk", right, f(V("T", 4, y)))
    right = ein("eVWYk,qQVRYW->eRkqQ", right, dbl(site[y]))
    return ein("eRkpP,eRkqQ->pqPQ", left, right).reshape(d * d, d * d)


def _iteration(A, B, chi, chip, eps, keys, *tensors):
    """One iteration (left, up, right, down) as a function of tensors, for checkpointing."""
    env = dict(zip(keys, tensors))
    for direction in O.MOVE_ORDER:
        move(env, direction, A, B, chi, chip, eps)
    return tuple(env[k] for k in keys)


def energy(env0, A, B, chi, iters, chip=None, eps=1e-12, checkpoint=False):
    """Mean Heisenberg bond energy after `iters` iterations (left, up, right, down)
    of the reduced-sequential move from the fixed environment env0 (numpy arrays).

    checkpoint=True keeps only each iteration's output environment for the
    backward pass and recomputes the iteration's intermediates there
    (torch.utils.checkpoint); the gradient is the same."""
    chip = chi if chip is None else chip
    keys = sorted(env0)
    tensors = tuple(torch.as_tensor(env0[k], dtype=DT) for k in keys)
    for _ in range(iters):
        if checkpoint:
            tensors = torch.utils.checkpoint.checkpoint(
                _iteration, A, B, chi, chip, eps, keys, *tensors, use_reentrant=False)
        else:
            tensors = _iteration(A, B, chi, chip, eps, keys, *tensors)
    env = dict(zip(keys, tensors))
    H = torch.as_tensor(O.heisenberg_bond(), dtype=DT)
    total = 0.0
    for bond, (r, x) in O.BONDS.items():
        rho = bond_rdm(env, A, B, r, x)
        total = total + torch.trace(rho @ H) / torch.trace(rho)
    return total / len(O.BONDS)


def energy_and_grad(env0, A, B, chi, iters, chip=None, eps=1e-12, checkpoint=False):
    """(E, dE/dA, dE/dB) as float and numpy arrays."""
    At = torch.tensor(A, dtype=DT, requires_grad=True)
    Bt = torch.tensor(B, dtype=DT, requires_grad=True)
    E = energy(env0, At, Bt, chi, iters, chip, eps, checkpoint)
    gA, gB = torch.autograd.grad(E, (At, Bt))
    return float(E.detach()), gA.numpy(), gB.numpy()
