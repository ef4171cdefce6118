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
