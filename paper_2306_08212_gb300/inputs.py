"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds no step of the CTM method: it only draws or writes down site
tensors.  Every generator is deterministic in its arguments.

* ``random_sites``: A, B with i.i.d. N(0, 1) real entries, each scaled to unit
  Frobenius norm (numpy ``default_rng(seed)``; A uses ``seed``, B ``seed + 1``).
* ``neel_sites``: a Neel-like product state (A = |up> (x) |0000>, B = |down> (x)
  |0000>) plus ``eps`` times N(0, 1) noise, then unit norm.
* ``product_sites``: D = 1 product state from two local spinors.
* ``ising_peps``: the PEPS whose norm network is the 2D Ising partition function.
"""
import numpy as np


def _unit(t):
    return t / np.linalg.norm(t)


def random_sites(d, D, seed=0):
    A = np.random.default_rng(seed).standard_normal((d, D, D, D, D))
    B = np.random.default_rng(seed + 1).standard_normal((d, D, D, D, D))
    return _unit(A), _unit(B)


def neel_sites(D, eps=1e-2, seed=0, d=2):
    A = np.zeros((d, D, D, D, D))
    B = np.zeros((d, D, D, D, D))
    A[0, 0, 0, 0, 0] = 1.0
    B[1, 0, 0, 0, 0] = 1.0
    rng = np.random.default_rng(seed)
    A = A + eps * rng.standard_normal(A.shape)
    B = B + eps * rng.standard_normal(B.shape)
    return _unit(A), _unit(B)


def product_sites(phi_a, phi_b):
    A = np.asarray(phi_a, float).reshape(-1, 1, 1, 1, 1)
    B = np.asarray(phi_b, float).reshape(-1, 1, 1, 1, 1)
    return _unit(A), _unit(B)


def ising_peps(beta):
    """A[s, u, l, d, r] = W[s,u] W[s,l] W[s,d] W[s,r] with W = sqrt(exp(beta/2 s s')).

    Each ket bond carries sum_u W[s,u] W[s',u] = exp(beta s s' / 2), each bra
    bond the same, and the physical leg ties ket and bra spins, so the norm
    network is the Ising partition function at inverse temperature beta
    (d = D = 2).  Also returns W: outer(W[0], W[0]) closes an outward leg on a
    fixed + spin, which selects the + phase above beta_c.
    """
    spins = np.array([1.0, -1.0])
    G = np.exp(0.5 * beta * np.outer(spins, spins))
    w, U = np.linalg.eigh(G)
    W = U @ np.diag(np.sqrt(w)) @ U.T
    A = np.einsum("su,sl,sd,sr->suldr", W, W, W, W)
    return A, W


def random_env_tensors(D, chi, seed=0):
    """Random real environment at bond dimension chi (16 tensors, clockwise legs).

    Corners are chi x chi, edges chi x D x D x chi; entries N(0, 1) scaled to
    unit norm.  Keyed ('C' | 'T', k, 'a' | 'b').
    """
    rng = np.random.default_rng(seed)
    env = {}
    for k in range(1, 5):
        for x in "ab":
            env[("C", k, x)] = _unit(rng.standard_normal((chi, chi)))
            env[("T", k, x)] = _unit(rng.standard_normal((chi, D, D, chi)))
    return env


def positive_env_tensors(D, c0, seed=0, terms=2, decay=0.0):
    """Random environment at bond dimension chi = c0^2 whose every tensor is a sum of
    `terms` ket (x) bra products (C = sum_t c_t (x) c_t, T = sum_t t_t (x) t_t, the
    boundary legs fused ket-slow), so that it is a positive boundary: every norm and
    density matrix it closes is a sum of squares, and energies lie in the spectrum of
    the operator.  With terms >= 2 the spectra carry no exact degeneracies of the
    Kronecker kind.  c_t, t_t ~ N(0, 1), their bond legs weighted by exp(-decay i)
    (index i of the leg; decay > 0 gives decaying spectra, like those of a converged
    environment); each sum scaled to unit norm.  Keyed ('C' | 'T', k, 'a' | 'b')."""
    rng = np.random.default_rng(seed)
    w = np.exp(-decay * np.arange(c0))
    env = {}
    for k in range(1, 5):
        for x in "ab":
            C = np.zeros((c0 * c0, c0 * c0))
            T = np.zeros((c0 * c0, D, D, c0 * c0))
            for _ in range(terms):
                c = rng.standard_normal((c0, c0)) * w[:, None] * w[None, :]
                t = rng.standard_normal((c0, D, c0)) * w[:, None, None] * w[None, None, :]
                C += np.einsum("ab,AB->aAbB", c, c).reshape(c0 * c0, c0 * c0)
                T += np.einsum("akb,AKB->aAkKbB", t, t).reshape(c0 * c0, D, D, c0 * c0)
            env[("C", k, x)] = _unit(C)
            env[("T", k, x)] = _unit(T)
    return env
