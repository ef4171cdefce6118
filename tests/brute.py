"""Brute-force contraction of small finite double-layer lattices (test helper).

Independent of the oracle: it builds the norm network of a rows x cols patch of
the checkerboard PEPS site by site, closes every outer leg with ``bnd``, and
contracts it row by row with plain tensordot.  Used to pin the oracle's exact
(untruncated) CTM moves.
"""
import numpy as np


def _site_tensor(A, open_phys):
    D = A.shape[1]
    if open_phys:
        a = np.einsum("puldr,PULDR->pPuUlLdDrR", A, A)
        return a.reshape(A.shape[0], A.shape[0], D * D, D * D, D * D, D * D)
    a = np.einsum("puldr,pULDR->uUlLdDrR", A, A)
    return a.reshape(D * D, D * D, D * D, D * D)


def finite_rdm(A, B, rows, cols, pair, a_parity=0, bnd=None):
    """rho[(i j), (i' j')] of two horizontally adjacent sites of a finite patch.

    Site (r, c) holds A when (r + c) % 2 == a_parity, else B.  ``pair`` is
    ((r, c), (r, c + 1)).  Every outer leg is closed with bnd (default identity).
    """
    D = A.shape[1]
    d = A.shape[0]
    if bnd is None:
        bnd = np.eye(D)
    e = bnd.reshape(D * D)
    opened = set(pair)
    # state legs: [v_0 .. v_{cols-1}, *phys]
    state = np.ones([1] * 0)
    state = e
    for _ in range(cols - 1):
        state = np.multiply.outer(state, e)
    nphys = 0
    for r in range(rows):
        # append the horizontal leg, closed on the left
        state = np.tensordot(state, e, axes=0)       # [v.., *phys, h]
        state = np.moveaxis(state, -1, cols)          # [v.., h, *phys]
        for c in range(cols):
            S = A if (r + c) % 2 == a_parity else B
            op = (r, c) in opened
            t = _site_tensor(S, op)
            if op:
                t = np.moveaxis(t, (0, 1), (4, 5))    # [U, L, Dn, R, p, P]
            out = np.tensordot(state, t, axes=([c, cols], [0, 1]))
            # out: [v (without c), *phys, Dn, R, (p, P)]
            nv = cols - 1
            k = nv + nphys
            out = np.moveaxis(out, k, c)              # Dn back to slot c
            out = np.moveaxis(out, k + 1, cols)       # R becomes the horizontal leg
            state = out
            if op:
                nphys += 2
        # close the horizontal leg on the right
        state = np.tensordot(state, e, axes=([cols], [0]))
    for c in range(cols):
        state = np.tensordot(state, e, axes=([0], [0]))
    # state: [p, P, q, Q] in the order the sites were opened (row-major)
    rho = state.reshape(d, d, d, d).transpose(0, 2, 1, 3)
    return rho.reshape(d * d, d * d)
