"""The allocation-free singular-value entry point against the regular one.

ctm_singular_values_noalloc serves callers that must not allocate device memory
during a call (a runtime that owns the device memory, or forbids cudaMalloc and
cudaFree after start-up): it works in a fixed scratch array inside the library.
Its output must equal what ctm_corner_spectrum returns for the same matrix set
as a corner of a context, on two calls in a row (the scratch keeps the previous
call's contents, so the second call checks that it starts clean).
"""
import numpy as np
import pytest

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


def test_noalloc_matches_corner_spectrum_twice(ctm):
    import torch
    A, B = I.random_sites(2, 2, 3)
    env = ctm.Env(A, B, 64)
    try:
        rng = np.random.default_rng(9)
        shapes = [(60, 45), (37, 64)]  # both orientations, ragged sizes
        for rows, cols in shapes:
            M = rng.standard_normal((rows, cols))
            env.set_tensor(0, 1, 0, M)
            ref = env.corner_spectrum(0)
            Md = torch.from_numpy(M).cuda()
            out = torch.full((min(rows, cols),), -1.0, dtype=torch.float64, device="cuda")
            rc = ctm.ctm_singular_values_noalloc(Md.data_ptr(), rows, cols, out.data_ptr())
            assert rc == ctm.OK
            got = out.cpu().numpy()
            assert got.shape == ref.shape
            np.testing.assert_allclose(got, ref, rtol=0, atol=TOL)
            # independent check of the values themselves
            sv = np.linalg.svd(M, compute_uv=False)
            np.testing.assert_allclose(got, sv / np.linalg.norm(sv), rtol=0, atol=TOL)
    finally:
        env.free()


def test_noalloc_rejects_sizes_beyond_the_scratch(ctm):
    import torch
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    Md = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert ctm.ctm_singular_values_noalloc(Md.data_ptr(), 2048, 1024, out.data_ptr()) == ctm.ERR_ARG
    assert ctm.ctm_singular_values_noalloc(Md.data_ptr(), 0, 4, out.data_ptr()) == ctm.ERR_ARG
