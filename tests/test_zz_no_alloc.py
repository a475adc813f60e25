"""bem_convolve_noalloc: the transform for callers that may not allocate.

Some callers cannot call cudaMalloc: hosts whose device memory belongs to a
caching allocator or arena they must not bypass, and loops that cannot afford
cudaMalloc's device-wide synchronisation.  This entry point gives them the FP64
transform u = A K*p with its scratch in a static device array.  These tests
call it through the C ABI and check it, on two calls in a row, against the
existing entry point bem_convolve (FP64) and against the oracle's direct sum
of Eq. 7, within the transform tolerance of the parity tests (1e-12 of the
field's maximum).  They also check that a call changes no device-memory
figure, and that a fresh process can use it before creating any handle.  The
file sorts last so that a run stopping at the first failure has run every
other test first.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from paper_1612_08395_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL = 1e-12  # of the field's maximum, as the FP64 transform parity tests


def _torus(n):
    return max(32, 1 << int(np.ceil(np.log2(2 * n))))


def _oracle_spectrum(oracle_mod, nx, ny, k):
    """FP64 real quarter of FFT(K) on the even Px x Py torus, as bem_spectrum lays it out."""
    px, py = _torus(nx), _torus(ny)
    Kq = oracle_mod.influence_quarter(k, 1.0 / nx, 1.0 / ny, px // 2 + 1, py // 2 + 1)
    return np.fft.fft2(oracle_mod.torus_kernel(Kq, py, px)).real[:py // 2 + 1, :px // 2 + 1].copy()


@pytest.mark.parametrize("nx,ny,k", [(64, 64, 0.3), (100, 37, -0.5), (16, 16, 0.5), (2, 2, -0.2),
                                     (256, 256, 0.6)])
def test_noalloc_matches_convolve_and_oracle_on_two_calls(bem_mod, oracle_mod, cuda_ok, nx, ny, k):
    import torch
    nu = 0.3
    A = oracle_mod.compliance(k, nu)
    Kq = oracle_mod.influence_quarter(k, 1.0 / nx, 1.0 / ny, nx, ny)
    with bem_mod.Handle(nx, ny, 1.0 / nx, 1.0 / ny, k, nu) as h:
        spec = torch.from_numpy(h.spectrum()).cuda()
        assert abs(h.info().compliance - A) <= 1e-14 * A
        for seed in (1, 2):
            p = I.random_pressure(nx, ny, seed=seed, density=0.6)
            ref = h.convolve(p, "fp64")
            pd = torch.from_numpy(p).cuda()
            ud = torch.full_like(pd, float("nan"))
            rc = bem_mod.convolve_noalloc(spec, nx, ny, A, pd, ud)
            torch.cuda.synchronize()
            assert rc == bem_mod.BEM_OK, bem_mod.load_library().bem_last_error()
            u = ud.cpu().numpy()
            scale = np.abs(ref).max()
            assert np.abs(u - ref).max() <= TOL * scale
            if nx * ny <= 128 * 128:
                uo = A * oracle_mod.convolve_direct(Kq, p)
                assert np.abs(u - uo).max() <= TOL * np.abs(uo).max()
            else:
                rng = np.random.Generator(np.random.PCG64(seed))
                idx = np.concatenate([rng.integers(0, nx * ny, 60), [0, nx - 1, nx * ny - 1]])
                uo = A * oracle_mod.convolve_direct_at(Kq, p, idx)
                assert np.abs(u.ravel()[idx] - uo).max() <= TOL * np.abs(uo).max()


def test_noalloc_changes_no_device_memory(bem_mod, oracle_mod, cuda_ok):
    import torch
    nx, ny, k = 96, 80, 0.2
    spec = torch.from_numpy(_oracle_spectrum(oracle_mod, nx, ny, k)).cuda()
    A = oracle_mod.compliance(k, 0.3)
    pd = torch.from_numpy(I.random_pressure(nx, ny, seed=5)).cuda()
    ud = torch.empty_like(pd)
    assert bem_mod.convolve_noalloc(spec, nx, ny, A, pd, ud) == bem_mod.BEM_OK  # warm-up (kernel loading)
    torch.cuda.synchronize()
    alloc0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
    assert bem_mod.convolve_noalloc(spec, nx, ny, A, pd, ud) == bem_mod.BEM_OK
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_in_fresh_process_before_any_handle(oracle_mod, cuda_ok, tmp_path):
    """A process that never creates a handle: the spectrum comes from a file (here
    the oracle's), and the first call does the device set-up itself."""
    nx, ny, k, nu = 256, 128, -0.3, 0.3
    spec = _oracle_spectrum(oracle_mod, nx, ny, k)
    A = oracle_mod.compliance(k, nu)
    p = I.random_pressure(nx, ny, seed=9, density=0.5)
    np.save(tmp_path / "spec.npy", spec)
    np.save(tmp_path / "p.npy", p)
    script = textwrap.dedent(f"""
        import sys, numpy as np, torch
        sys.path.insert(0, {ROOT!r})
        from paper_1612_08395_gb300 import build, bem
        build.build()
        spec = torch.from_numpy(np.load({str(tmp_path / 'spec.npy')!r})).cuda()
        pd = torch.from_numpy(np.load({str(tmp_path / 'p.npy')!r})).cuda()
        out = []
        for _ in range(2):
            ud = torch.full_like(pd, float("nan"))
            rc = bem.convolve_noalloc(spec, {nx}, {ny}, {A!r}, pd, ud)
            torch.cuda.synchronize()
            assert rc == bem.BEM_OK, bem.load_library().bem_last_error()
            out.append(ud.cpu().numpy())
        np.save({str(tmp_path / 'u.npy')!r}, np.stack(out))
    """)
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    u = np.load(tmp_path / "u.npy")
    Kq = oracle_mod.influence_quarter(k, 1.0 / nx, 1.0 / ny, nx, ny)
    rng = np.random.Generator(np.random.PCG64(4))
    idx = np.concatenate([rng.integers(0, nx * ny, 80), [0, nx - 1, nx * ny - 1]])
    uo = A * oracle_mod.convolve_direct_at(Kq, p, idx)
    for call in u:
        assert np.abs(call.ravel()[idx] - uo).max() <= TOL * np.abs(uo).max()


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
