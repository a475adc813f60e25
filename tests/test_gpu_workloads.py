"""Full-size workloads and the paper's invariants on the GPU path.

- 4096 x 4096 seeded self-affine rough surface (the 4096^2 non-adhesive workload):
  complementarity at sampled elements, evaluated with the oracle's influence table
  and direct sum of Eq. 7 (a property of the solution that holds at any size).
- Mesh independence of the adhesive pull-off of a paraboloid (Sec. 3.2, Fig. 7):
  256^2 and 1024^2 grids give the same force-depth behaviour.
"""
import numpy as np
import pytest

from paper_1612_08395_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_rough_surface_4096_complementarity(bem_mod, oracle_mod, cuda_ok):
    n, k, nu = 4096, 0.3, 0.3
    dx = 1.0 / n
    h, zrms = I.rough_self_affine(n, hurst=0.8, q1_over_q0=256.0, rms_slope=0.1, seed=1612)
    d = zrms
    p = np.empty((n, n))
    with bem_mod.Handle(n, n, dx, dx, k, nu) as hd:
        res, rc = hd.solve(h, d, pressure_out=p, precision="fp32_refine")
    assert rc == bem_mod.BEM_OK
    frac = res.contact_count / n / n
    assert 1e-3 < frac < 0.5
    assert p.min() >= 0.0
    assert res.force == pytest.approx(p.sum() * dx * dx, rel=1e-12)
    # sampled complementarity with the oracle's operator
    A = oracle_mod.compliance(k, nu)
    Kq = oracle_mod.influence_quarter(k, dx, dx, n, n, rel_tol=1e-13)
    rng = np.random.Generator(np.random.PCG64(7))
    flat = p.ravel()
    on = np.flatnonzero(flat > 0)
    off = np.flatnonzero(flat == 0)
    idx = np.concatenate([rng.choice(on, 40, replace=False), rng.choice(off, 40, replace=False)])
    g = A * oracle_mod.convolve_direct_at(Kq, p, idx) + h.ravel()[idx] - d
    assert np.abs(g[:40]).max() <= 1e-8 * d
    assert g[40:].min() >= -1e-8 * d


def test_adhesive_mesh_independence(bem_mod, oracle_mod, cuda_ok):
    from oracle import closed_forms as CF
    k, nu, R, gam, d0 = 0.5, 0.3, 1.0, 1e-3, 0.01
    a0 = CF.hertz_radius(d0, k, R)
    aa = np.linspace(1e-3, a0, 4000)
    Fmin = min(CF.jkr_force(x, k, nu, R, gam) for x in aa)
    dmin = min(CF.jkr_depth(x, k, nu, R, gam) for x in aa)
    steps = np.concatenate([[d0], np.linspace(d0, 1.2 * dmin, 201)[1:]])
    out = {}
    for n in (256, 1024):
        with bem_mod.Handle(n, n, 1.0 / n, 1.0 / n, k, nu) as hd:
            res, rc = hd.sweep(I.paraboloid(n, R), steps, dgamma=gam, precision="fp32")
        F = np.array([r.force for r in res])
        cnt = np.array([r.contact_count for r in res])
        last = np.flatnonzero(cnt > 0).max()
        out[n] = (F, F.min(), steps[last])
    # the two meshes agree (Fig. 7) and follow the JKR-type closed form
    assert out[256][1] == pytest.approx(out[1024][1], rel=0.03)
    assert out[256][2] == pytest.approx(out[1024][2], rel=0.03)
    for n in out:
        assert out[n][1] == pytest.approx(Fmin, rel=0.05)
        assert out[n][2] == pytest.approx(dmin, rel=0.05)
    # force curves agree step by step on the stable branch, up to the force minimum
    # (beyond it the contact shrinks to a few elements before it snaps off)
    both = min(int(np.argmin(out[256][0])), int(np.argmin(out[1024][0])))
    assert np.abs(out[256][0][:both] - out[1024][0][:both]).max() <= 0.03 * abs(Fmin)
