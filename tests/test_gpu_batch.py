"""Batched independent states (uneven D, chi = 2 D^2) give
the same results as advancing each state alone."""
import numpy as np
import pytest

from oracle import ctm_oracle as O
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


def _make(ctm, torch, Ds):
    envs = []
    for i, D in enumerate(Ds):
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            A, B = I.random_sites(2, D, 100 + i)
            envs.append(ctm.Env(A, B, 2 * D * D, precision="tf32"))
    return envs


def _observe(envs):
    H = O.heisenberg_bond()
    return [([e.expect_bond(b, H) for b in range(4)], e.corner_spectra()) for e in envs]


def test_batch_equals_individual_moves(ctm):
    import torch
    Ds = [3, 5, 6, 4]
    solo = _make(ctm, torch, Ds)
    many = _make(ctm, torch, Ds)
    batch = ctm.Batch(many)
    try:
        for _ in range(3):
            for d in O.MOVE_ORDER:
                batch.move(d, "reduced_sequential")
                for e in solo:
                    e.move(d, "reduced_sequential")
        torch.cuda.synchronize()
        for (e0, s0), (e1, s1) in zip(_observe(solo), _observe(many)):
            np.testing.assert_allclose(e1, e0, rtol=0, atol=1e-12)
            for a, b in zip(s0, s1):
                np.testing.assert_allclose(b, a, rtol=0, atol=1e-12)
    finally:
        batch.free()
        for e in solo + many:
            e.free()


def test_32_uneven_states_against_the_oracle_and_their_solo_runs(ctm):
    """32 states with D drawn uniformly from {3..7} (seed 0) and chi = 2 D^2 in TF32, all
    four moves of each state through one batch (one CUDA graph launch per direction once
    warm).  The state with the smallest D is compared with the oracle after the same
    moves (TF32 error bound), and the smallest and largest states with their solo runs."""
    import time

    import torch
    rng = np.random.default_rng(0)
    Ds = [int(v) for v in rng.integers(3, 8, size=32)]
    many = _make(ctm, torch, Ds)
    batch = ctm.Batch(many)
    i_small, i_large = int(np.argmin(Ds)), int(np.argmax(Ds))
    solo = []
    for k in (i_small, i_large):  # the same sites (seeds) as those batch members
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            A, B = I.random_sites(2, Ds[k], 100 + k)
            solo.append(ctm.Env(A, B, 2 * Ds[k] ** 2, precision="tf32"))
    try:
        iters = 3
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(iters):
            for d in O.MOVE_ORDER:
                batch.move(d, "reduced_sequential")
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        print(f"32 states, D={sorted(Ds)}: {4 * iters * 32 / dt:.1f} state-moves/s "
              f"(first iteration captures the graphs)")
        for _ in range(iters):
            for d in O.MOVE_ORDER:
                for e in solo:
                    e.move(d, "reduced_sequential")
        torch.cuda.synchronize()
        (e0, s0), (e1, s1) = _observe([solo[0]])[0], _observe([many[i_small]])[0]
        np.testing.assert_allclose(e1, e0, rtol=0, atol=1e-12)
        (e0, s0), (e1, s1) = _observe([solo[1]])[0], _observe([many[i_large]])[0]
        np.testing.assert_allclose(e1, e0, rtol=0, atol=1e-12)
        # the smallest state against the oracle
        D = Ds[i_small]
        chi = 2 * D * D
        A, B = I.random_sites(2, D, 100 + i_small)
        env = O.init_env(A, B, chi)
        for _ in range(iters):
            for d in O.MOVE_ORDER:
                O.move(env, d, A, B, chi, chi, "reduced_sequential")
        H = O.heisenberg_bond()
        ref = [O.expect_bond(env, A, B, b, H) for b in range(4)]
        got = [many[i_small].expect_bond(b, H) for b in range(4)]
        de = max(abs(a - b) for a, b in zip(ref, got))
        print(f"batched D={D} chi={chi} TF32 vs oracle after {iters} iterations: |dE_bond| = {de:.2e}")
        # On small random states the reduced-sequential iteration does not settle: its
        # bond energies wander by a few 1e-4 from one iteration to the next (the band
        # shrinks as chi grows, measured with the oracle alone), so a trajectory that
        # starts from projectors of a different precision stays within that band only.
        assert de < 5e-3
    finally:
        batch.free()
        for e in solo + many:
            e.free()
