"""bem_convolve_noalloc: the transform for callers that may not allocate.

Callers that cannot call cudaMalloc (code running under stream capture, hosts
whose device memory belongs to a pool, loops that cannot afford cudaMalloc's
device-wide synchronisation) use this entry point; its scratch is a static
device array.  These tests check it through the C ABI against bem_convolve's
FP64 transform, within the transform tolerance of the parity tests (1e-12 of
the field's maximum), on two calls in a row.  The file sorts last so that a
run stopping at the first failure has run every other test first.
"""
import numpy as np
import pytest

from paper_1612_08395_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nx,ny,k", [(64, 64, 0.3), (100, 37, -0.5), (256, 256, 0.6)])
def test_noalloc_matches_convolve_on_two_calls(bem_mod, cuda_ok, nx, ny, k):
    import torch
    with bem_mod.Handle(nx, ny, 1.0 / nx, 1.0 / ny, k, 0.3) as h:
        spec = torch.from_numpy(h.spectrum()).cuda()
        A = h.info().compliance
        for seed in (1, 2):
            p = I.random_pressure(nx, ny, seed=seed, density=0.6)
            ref = h.convolve(p, "fp64")
            pd = torch.from_numpy(p).cuda()
            ud = torch.full_like(pd, float("nan"))
            rc = bem_mod.convolve_noalloc(spec, nx, ny, A, pd, ud)
            torch.cuda.synchronize()
            assert rc == bem_mod.BEM_OK, bem_mod.load_library().bem_last_error()
            u = ud.cpu().numpy()
            assert np.abs(u - ref).max() <= 1e-12 * np.abs(ref).max()


def test_noalloc_rejects_bad_calls(bem_mod, cuda_ok):
    import torch
    n = 16
    with bem_mod.Handle(n, n, 1.0 / n, 1.0 / n, 0.2, 0.3) as h:
        spec = torch.from_numpy(h.spectrum()).cuda()
        A = h.info().compliance
    big = torch.zeros((257, 257), dtype=torch.float64, device="cuda")
    assert bem_mod.convolve_noalloc(spec, 257, 257, A, big, big) == bem_mod.BEM_EINVAL
    assert b"256" in bem_mod.load_library().bem_last_error()
    ph = np.zeros((n, n))
    ud = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    assert bem_mod.convolve_noalloc(spec, n, n, A, ph, ud) == bem_mod.BEM_EINVAL
