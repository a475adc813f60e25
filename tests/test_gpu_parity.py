"""CUDA path vs the FP64 oracle, element by element (GPU required).

Every input is seeded and synthetic; expected values come only from oracle/.
Tolerances: FP64 path 1e-10 relative (pressures), 1e-12 (influence table,
spectrum, transform); FP32 transform 2e-6 of the field's max, FP32 pressures
1e-5 relative L2; contact counts exact.
"""
import math

import numpy as np
import pytest

from paper_1612_08395_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def relL2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def torus_sizes(nx, ny):
    px = max(32, 1 << int(math.ceil(math.log2(2 * nx))))
    py = max(32, 1 << int(math.ceil(math.log2(2 * ny))))
    return px, py


# ------------------------------------------------------------------ a1
@pytest.mark.parametrize("nx,ny,aspect", [(16, 16, 1), (24, 40, 1), (64, 64, 1), (7, 5, 1), (8, 40, 17),
                                          (40, 8, 17)])
@pytest.mark.parametrize("k", [-0.9, -0.5, 0.0, 0.3, 0.9])
def test_influence_table(bem_mod, oracle_mod, cuda_ok, nx, ny, aspect, k):
    # aspect > 1: elements `aspect` times longer in x (ny = 40) or in y (nx = 40).
    # At k = 0.9 the oracle's adaptive cubature of the self-term of such an
    # element, (a^2+b^2)^-0.95 over a 17:1 rectangle, does not converge (it
    # returns inf), so that case is left out.
    if aspect > 1 and k > 0.5:
        pytest.skip("oracle cubature of a 17:1 self-term at k = 0.9 does not converge")
    dx, dy = 1.0 / nx, 1.0 / ny
    if aspect > 1:
        dx, dy = (aspect / 136.0, 1 / 136.0) if ny > nx else (1 / 136.0, aspect / 136.0)
    with bem_mod.Handle(nx, ny, dx, dy, k, 0.3) as h:
        Kg = h.influence_table()
    px, py = torus_sizes(nx, ny)
    Ko = oracle_mod.influence_quarter(k, dx, dy, px // 2 + 1, py // 2 + 1)
    assert Kg.shape == Ko.shape
    np.testing.assert_allclose(Kg, Ko, rtol=1e-12, atol=0)


@pytest.mark.parametrize("nx,ny", [(16, 16), (24, 40), (64, 64)])
@pytest.mark.parametrize("k", [-0.9, 0.0, 0.5])
def test_spectrum(bem_mod, oracle_mod, cuda_ok, nx, ny, k):
    dx, dy = 1.0 / nx, 1.0 / ny
    px, py = torus_sizes(nx, ny)
    with bem_mod.Handle(nx, ny, dx, dy, k, 0.3) as h:
        Sg = h.spectrum()
    Ko = oracle_mod.influence_quarter(k, dx, dy, px // 2 + 1, py // 2 + 1)
    So = np.fft.fft2(oracle_mod.torus_kernel(Ko, py, px)).real[:py // 2 + 1, :px // 2 + 1]
    assert np.abs(Sg - So).max() <= 1e-12 * np.abs(So).max()
    assert Sg.min() > 0


# ------------------------------------------------------------------ a2-a4
@pytest.mark.parametrize("nx,ny", [(8, 8), (33, 17), (64, 64), (100, 37), (2, 2), (128, 128)])
@pytest.mark.parametrize("k", [-0.6, 0.4])
def test_convolution(bem_mod, oracle_mod, cuda_ok, nx, ny, k):
    dx, dy = 1.0 / nx, 1.0 / ny
    nu = 0.3
    p = I.random_pressure(nx, ny, seed=nx * 1000 + ny, density=0.7)
    Ko = oracle_mod.influence_quarter(k, dx, dy, nx, ny)
    uo = oracle_mod.compliance(k, nu) * oracle_mod.convolve_direct(Ko, p)
    with bem_mod.Handle(nx, ny, dx, dy, k, nu) as h:
        u64 = h.convolve(p, "fp64")
        u32 = h.convolve(p, "fp32")
    scale = np.abs(uo).max()
    assert np.abs(u64 - uo).max() <= 1e-12 * scale
    assert np.abs(u32 - uo).max() <= 2e-6 * scale


def test_convolution_device_pointers(bem_mod, oracle_mod, cuda_ok):
    import torch
    nx = ny = 48
    p = I.random_pressure(nx, ny, seed=11)
    with bem_mod.Handle(nx, ny, 1 / nx, 1 / ny, 0.2, 0.3) as h:
        uh = h.convolve(p, "fp64")
        pd = torch.from_numpy(p).cuda()
        ud = h.convolve(pd, "fp64")
        torch.cuda.synchronize()
    np.testing.assert_array_equal(ud.cpu().numpy(), uh)


@pytest.mark.parametrize("k", [0.3, -0.5])
def test_convolution_full_size_sampled(bem_mod, oracle_mod, cuda_ok, k):
    # 2048 x 2048 (the 2048^2 workload's transform) on 64 sampled outputs.
    n = 2048
    dx = 1.0 / n
    nu = 0.3
    p = np.maximum(0.0, 1.0 - (I.radius_grid(n, n, dx) / 0.3) ** 2) \
        + 0.1 * I.random_pressure(n, n, seed=7, density=0.01)
    rng = np.random.Generator(np.random.PCG64(3))
    idx = np.concatenate([rng.integers(0, n * n, 60), [0, n - 1, n * n - 1, n * (n // 2) + n // 2]])
    Ko = oracle_mod.influence_quarter(k, dx, dx, n, n)
    uo = oracle_mod.compliance(k, nu) * oracle_mod.convolve_direct_at(Ko, p, idx)
    with bem_mod.Handle(n, n, dx, dx, k, nu) as h:
        u64 = h.convolve(p, "fp64").ravel()[idx]
        u32 = h.convolve(p, "fp32").ravel()[idx]
    scale = np.abs(uo).max()
    assert np.abs(u64 - uo).max() <= 1e-11 * scale
    assert np.abs(u32 - uo).max() <= 5e-6 * scale


# ------------------------------------------------------------------ a5-a8: non-adhesive
@pytest.fixture(scope="module")
def config1_oracle(oracle_mod):
    n, k, nu, d = 64, 0.5, 0.3, 0.01
    dx = 1.0 / n
    A = oracle_mod.compliance(k, nu)
    Kq = oracle_mod.influence_quarter(k, dx, dx, n, n)
    h = I.paraboloid(n)
    res = oracle_mod.pk_solve(A, oracle_mod.DirectConvolver(Kq, n, n), h, d, tol=1e-12)
    return dict(n=n, k=k, nu=nu, d=d, h=h, p=res.p, it=res.iterations)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-4), ("fp32_refine", 1e-10)])
def test_config1_solve(bem_mod, cuda_ok, config1_oracle, prec, tol):
    c = config1_oracle
    n = c["n"]
    p = np.empty((n, n))
    with bem_mod.Handle(n, n, 1 / n, 1 / n, c["k"], c["nu"]) as h:
        res, rc = h.solve(c["h"], c["d"], pressure_out=p, precision=prec,
                          tol=1e-12 if prec == "fp64" else 0.0)
    assert rc == bem_mod.BEM_OK
    assert relL2(p, c["p"]) <= tol
    assert res.contact_count == int((c["p"] > 0).sum())
    assert res.force == pytest.approx((c["p"].sum()) / n / n, rel=tol * 10)


@pytest.mark.parametrize("k", [-0.5, 0.5])
def test_flat_punch_solve(bem_mod, oracle_mod, cuda_ok, k):
    n, nu, a, d = 64, 0.3, 0.2, 0.01
    dx = 1.0 / n
    hprof = I.flat_punch(n, a)
    A = oracle_mod.compliance(k, nu)
    ref = oracle_mod.pk_solve(A, oracle_mod.FFTConvolver(
        oracle_mod.influence_quarter(k, dx, dx, n + 1, n + 1), n, n), hprof, d, tol=1e-12).p
    p = np.empty((n, n))
    with bem_mod.Handle(n, n, dx, dx, k, nu) as h:
        res, rc = h.solve(hprof, d, pressure_out=p, precision="fp64", tol=1e-12)
    assert relL2(p, ref) <= 1e-10
    assert res.contact_count == int((ref > 0).sum())


def test_nonsquare_ragged_solve(bem_mod, oracle_mod, cuda_ok):
    nx, ny, k, nu, d = 45, 29, -0.2, 0.25, 0.012
    dx, dy = 1.0 / 48, 1.0 / 32
    x = I.centres(nx, dx)
    y = I.centres(ny, dy)
    hprof = (x[None, :] ** 2 + 0.7 * y[:, None] ** 2) / 2.0
    A = oracle_mod.compliance(k, nu)
    Kq = oracle_mod.influence_quarter(k, dx, dy, nx, ny)
    ref = oracle_mod.pk_solve(A, oracle_mod.DirectConvolver(Kq, ny, nx), hprof, d, tol=1e-12).p
    p = np.empty((ny, nx))
    with bem_mod.Handle(nx, ny, dx, dy, k, nu) as h:
        res, rc = h.solve(hprof, d, pressure_out=p, precision="fp64", tol=1e-12)
    assert relL2(p, ref) <= 1e-10
    assert res.contact_count == int((ref > 0).sum())


def test_separated_and_degenerate(bem_mod, cuda_ok):
    n = 16
    with bem_mod.Handle(n, n, 1 / n, 1 / n, 0.3, 0.3) as h:
        p = np.empty((n, n))
        res, rc = h.solve(I.paraboloid(n) + 0.5, 0.1, pressure_out=p, precision="fp64")
        assert rc == bem_mod.BEM_OK and res.force == 0 and res.contact_count == 0
        assert (p == 0).all()
        # a 2 x 2 grid works too
    with bem_mod.Handle(2, 2, 0.5, 0.5, 0.3, 0.3) as h:
        res, rc = h.solve(np.zeros((2, 2)), 0.01, precision="fp64")
        assert rc == bem_mod.BEM_OK and res.contact_count == 4


def test_deterministic(bem_mod, cuda_ok):
    n = 96
    prof = I.paraboloid(n)
    outs = []
    with bem_mod.Handle(n, n, 1 / n, 1 / n, -0.3, 0.3) as h:
        for _ in range(2):
            p = np.empty((n, n))
            h.solve(prof, 0.015, pressure_out=p, precision="fp32")
            outs.append(p)
    np.testing.assert_array_equal(outs[0], outs[1])


@pytest.mark.parametrize("k,nu,shape", [(-0.5, 0.5, "paraboloid"), (0.5, 0.3, "flat")])
def test_config2_sweep_512(bem_mod, oracle_mod, cuda_ok, k, nu, shape):
    # 512 x 512 sweep (warm-started steps), sampled steps vs the oracle's FFT mode.
    n = 512
    dx = 1.0 / n
    prof = I.paraboloid(n) if shape == "paraboloid" else I.flat_punch(n, 0.2)
    ds = 0.02 * np.arange(1, 51) / 50
    A = oracle_mod.compliance(k, nu)
    conv = oracle_mod.FFTConvolver(oracle_mod.influence_quarter(k, dx, dx, n + 1, n + 1), n, n)
    check = [9, 49]
    with bem_mod.Handle(n, n, dx, dx, k, nu) as h:
        # plain FP32 has a rounding floor of 5e-5..1.5e-4 at k = -0.5 (conditioning x
        # FP32 transform error); the refined path carries the 1e-5 bar with margin
        for prec, tol in (("fp64", 1e-10), ("fp32_refine", 1e-10), ("fp32", 3e-4)):
            for j in check:
                p = np.empty((n, n))
                res, rc = h.sweep(prof, ds[:j + 1], final_pressure=p, precision=prec,
                                  tol={"fp64": 1e-12, "fp32": 1e-8}.get(prec, 0.0))
                ref = oracle_mod.pk_solve(A, conv, prof, ds[j], tol=1e-12).p
                assert relL2(p, ref) <= tol, (prec, j)
                Fs = [r.force for r in res]
                assert np.all(np.diff(Fs) > 0)


# ------------------------------------------------------------------ a7: adhesive
@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_adhesive_paraboloid_sweep(bem_mod, oracle_mod, cuda_ok, prec):
    n, k, nu, gam, d0 = 64, 0.5, 0.3, 1e-3, 0.01
    dx = 1.0 / n
    prof = I.paraboloid(n)
    A = oracle_mod.compliance(k, nu)
    conv = oracle_mod.DirectConvolver(oracle_mod.influence_quarter(k, dx, dx, n, n), n, n)
    steps = np.linspace(d0, -0.04, 61)
    out, p_ref, S_ref = oracle_mod.adhesive_unload(A, conv, prof, d0, steps[1:],
                                                   oracle_mod.p_crit(k, nu, gam, dx), dx * dx,
                                                   tol_pk=1e-12, tol_cg=1e-13)
    p = np.empty((n, n))
    with bem_mod.Handle(n, n, dx, dx, k, nu) as h:
        res, rc = h.sweep(prof, steps, dgamma=gam, final_pressure=p, precision=prec, tol=1e-12)
    for o, r in zip(out, res[1:]):
        assert r.contact_count == o["count"], (o["d"], r.contact_count, o["count"])
        assert r.force == pytest.approx(o["force"], rel=1e-8, abs=1e-14)
    assert relL2(p, p_ref) <= 1e-9 or (p_ref == 0).all() and (p == 0).all()


def test_adhesive_rejects_bad_input(bem_mod, cuda_ok):
    n = 16
    with bem_mod.Handle(n, n, 1 / n, 1 / 8, 0.3, 0.3) as h:
        with pytest.raises(bem_mod.BemError) as e:
            h.sweep(I.paraboloid(n), [0.01, 0.0], dgamma=1e-3)
        assert e.value.code == bem_mod.BEM_EINVAL
    with bem_mod.Handle(n, n, 1 / n, 1 / n, 0.3, 0.3) as h:
        with pytest.raises(bem_mod.BemError) as e:
            h.sweep(I.paraboloid(n), [0.01, 0.02], dgamma=1e-3)
        assert e.value.code == bem_mod.BEM_EINVAL


# ------------------------------------------------------------------ work accounting
def test_pass_work_full_torus_and_box(bem_mod, cuda_ok):
    """bem_pass_work: a flat indenter pressed in everywhere keeps the full torus, so
    pass B moves W (in and out) and the spectrum quarter; an adhesive paraboloid's
    fixed-set solves run on the contact box's smaller torus and move less."""
    n = 64
    dx = 1.0 / n
    px, py = torus_sizes(n, n)
    M = px // 2
    full_b = 2 * 8 * (M + 1) * n + 4 * (M + 1) * (py // 2 + 1)
    with bem_mod.Handle(n, n, dx, dx, 0.3, 0.3) as h:
        h.pass_times(reset=True)
        res, rc = h.solve(np.zeros((n, n)), 1e-3, precision="fp32", time_passes=True)
        (ba, bb, bc), (fa, fb, fc) = h.pass_work()
        ms, cnt, cnt_cg = h.pass_times(reset=True)
        assert cnt > 0 and cnt_cg == 0
        assert bb == full_b
        assert ba == 16 * n * n + 8 * (M + 1) * n and bc == 12 * n * n + 8 * (M + 1) * n
        steps = np.linspace(0.01, -0.01, 21)
        h.sweep(I.paraboloid(n), steps, dgamma=1e-3, precision="fp32", time_passes=True)
        (ba2, bb2, bc2), _ = h.pass_work()
        ms2, cnt2, cnt_cg2 = h.pass_times(reset=True)
        assert cnt_cg2 > 0
        assert bb2 < 0.5 * full_b
