"""Mixed precision (TF32 / BF16 contractions, FP64 factorisations) against the
FP64 path on gauge-invariant outputs.  The bound is loose by design: it states
the error, it does not hide a wrong kernel (a layout error gives O(1) errors).
Measured errors are printed (pytest -s)."""
import numpy as np
import pytest

from oracle import ctm_oracle as O
from paper_2306_08212_gb300 import inputs as I

pytestmark = pytest.mark.gpu

BOUND = {"tf32": 2e-3, "bf16": 2e-2}


@pytest.fixture(scope="module")
def ctm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_08212_gb300 import ctm as C
    C.load()
    return C


def _run(ctm, A, B, chi, prec, iters):
    g = ctm.Env(A, B, chi, precision=prec)
    try:
        for _ in range(iters):
            for d in O.MOVE_ORDER:
                g.move(d, "reduced_sequential")
        H = O.heisenberg_bond()
        return [g.expect_bond(b, H) for b in range(4)], g.corner_spectra()
    finally:
        g.free()


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_mixed_precision_error_vs_fp64(ctm, prec):
    A, B = I.neel_sites(4, eps=1e-2, seed=0)
    e64, s64 = _run(ctm, A, B, 64, "fp64", 2)
    em, sm = _run(ctm, A, B, 64, prec, 2)
    de = max(abs(a - b) for a, b in zip(e64, em))
    ds = max(np.abs(a[:16] - b[:16]).max() for a, b in zip(s64, sm))
    print(f"{prec}: max |dE_bond| = {de:.3e}, max |ds| (top 16) = {ds:.3e}")
    assert de < BOUND[prec]
    assert ds < BOUND[prec]


def test_graph_replay_matches_eager(ctm):
    """Steady-state moves replayed from CUDA graphs (context on a side stream)
    give the same results as eager execution (context on the default stream)."""
    import torch
    A, B = I.random_sites(2, 4, 2)
    H = O.heisenberg_bond()
    res = []
    for use_side in (False, True):
        stream = torch.cuda.Stream() if use_side else torch.cuda.default_stream()
        with torch.cuda.stream(stream):
            g = ctm.Env(A, B, 64, precision="tf32")
            try:
                for _ in range(3):
                    for d in O.MOVE_ORDER:
                        g.move(d, "reduced_sequential")
                res.append(([g.expect_bond(b, H) for b in range(4)], g.corner_spectra()))
            finally:
                g.free()
    (e0, s0), (e1, s1) = res
    np.testing.assert_allclose(e1, e0, rtol=0, atol=1e-12)
    for a, b in zip(s0, s1):
        np.testing.assert_allclose(b, a, rtol=0, atol=1e-12)
