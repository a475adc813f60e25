"""Regression tests after the paper's Figs. 8 and 10 (Sec. 3.2), on the GPU path.

Fig. 8: adhesive pull-off of a paraboloid from graded half-spaces of several
k and R/c0 on a 512 x 512 grid.  The force minimum and the last contact depth
follow the JKR-type closed form built from Eqs. 15, 16 and 25 (oracle
closed_forms.jkr_force / jkr_depth).  The contact is preloaded without
adhesion to the radius a0 and can only shrink afterwards, so the comparison is
with the minima over a <= a0.

The same closed form at 2048 x 2048 on the load-unload sweep (k = 0.3, preload
d0 = 0.02, 400 unloading steps of 1.1e-4): force minimum and jump-off depth.

Fig. 10: adhesive pull-off of a flat square punch whose edges make 0, 15, 30 and
45 degrees with the grid (k = 0.3, 512 x 512): the macroscopic curve does not
depend on the orientation -- pull-off force, jump-off depth and initial contact
area agree across orientations.
"""
import numpy as np
import pytest

from paper_1612_08395_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def pull_off(bem_mod, n, k, R, c0, nu=0.3, gam=1e-3, a0=0.15, nsteps=481):
    """(simulated force minimum, last contact depth, closed-form minima over a <= a0)."""
    from oracle import closed_forms as CF
    d0 = CF.hertz_depth(a0, k, R)
    aa = np.linspace(1e-3, a0, 4000)
    Fmin = min(CF.jkr_force(x, k, nu, R, gam, 1.0, c0) for x in aa)
    dmin = min(CF.jkr_depth(x, k, nu, R, gam, 1.0, c0) for x in aa)
    steps = np.concatenate([[d0], np.linspace(d0, 1.2 * dmin, nsteps)[1:]])
    with bem_mod.Handle(n, n, 1.0 / n, 1.0 / n, k, nu, 1.0, c0) as hd:
        res, rc = hd.sweep(I.paraboloid(n, R), steps, dgamma=gam, precision="fp32")
    assert rc == bem_mod.BEM_OK
    F = np.array([r.force for r in res])
    cnt = np.array([r.contact_count for r in res])
    assert cnt[-1] == 0  # pulled off within the sweep
    return F.min(), steps[np.flatnonzero(cnt > 0).max()], Fmin, dmin


# k < 0 sharpens the edge singularity of the adhesive stress (exponent -(1-k)/2) and
# the discrete pull-off converges more slowly: that family runs on 1024^2
@pytest.mark.parametrize("k,R,c0,n", [(-0.5, 1.0, 1.0, 1024), (0.0, 0.5, 1.0, 512), (0.3, 2.0, 1.0, 512),
                                      (0.5, 1.0, 0.5, 512), (0.7, 1.0, 2.0, 512)])
def test_fig8_graded_families_follow_jkr(bem_mod, cuda_ok, k, R, c0, n):
    F, d, Fmin, dmin = pull_off(bem_mod, n, k, R, c0)
    assert F == pytest.approx(Fmin, rel=0.05)
    assert d == pytest.approx(dmin, rel=0.05)


def test_fig8_pull_off_converges_with_mesh(bem_mod, cuda_ok):
    # k = -0.5: the distance to the closed form shrinks with every refinement
    errs = []
    for n in (256, 512, 1024):
        F, d, Fmin, dmin = pull_off(bem_mod, n, -0.5, 1.0, 1.0)
        errs.append((abs(F / Fmin - 1), abs(d / dmin - 1)))
    for q in range(2):
        assert errs[0][q] > errs[1][q] > errs[2][q]
    assert errs[2][0] < 0.03 and errs[2][1] < 0.03


def test_pull_off_2048_follows_jkr(bem_mod, cuda_ok):
    # the 2048 x 2048 load-unload sweep (k = 0.3, preload d0 = 0.02, 400 unloading steps
    # of 1.1e-4): the contact starts at the Hertz radius a0 and shrinks, so the force
    # minimum is the closed form's minimum over a <= a0 (at a0 here) and the last contact
    # depth the closed form's jump-off depth
    from oracle import closed_forms as CF
    n, k, nu, R, gam, d0 = 2048, 0.3, 0.3, 1.0, 1e-3, 0.02
    a0 = CF.hertz_radius(d0, k, R)
    aa = np.linspace(1e-3, a0, 4000)
    Fmin = min(CF.jkr_force(x, k, nu, R, gam) for x in aa)
    dmin = min(CF.jkr_depth(x, k, nu, R, gam) for x in aa)
    steps = np.array([d0] + [d0 - 1.1e-4 * j for j in range(1, 401)])
    with bem_mod.Handle(n, n, 1.0 / n, 1.0 / n, k, nu) as hd:
        res, rc = hd.sweep(I.paraboloid(n, R), steps, dgamma=gam, precision="fp32")
    assert rc == bem_mod.BEM_OK
    F = np.array([r.force for r in res])
    cnt = np.array([r.contact_count for r in res])
    assert cnt[-1] == 0
    # preload: graded Hertz (Eqs. 15, 16)
    assert F[0] == pytest.approx(CF.hertz_force(a0, k, nu, R), rel=1e-3)
    assert F.min() == pytest.approx(Fmin, rel=0.01)
    assert steps[np.flatnonzero(cnt > 0).max()] == pytest.approx(dmin, abs=1.1e-4)


def test_fig10_square_punch_orientation_independent(bem_mod, cuda_ok):
    n, k, nu, gam, side = 512, 0.3, 0.3, 1e-3, 0.3
    steps = np.linspace(0.005, -0.06, 261)
    out = {}
    for ang in (0.0, 15.0, 30.0, 45.0):
        prof = I.square_punch(n, side, ang)
        with bem_mod.Handle(n, n, 1.0 / n, 1.0 / n, k, nu) as hd:
            res, rc = hd.sweep(prof, steps, dgamma=gam, precision="fp32")
        assert rc == bem_mod.BEM_OK
        F = np.array([r.force for r in res])
        cnt = np.array([r.contact_count for r in res])
        assert cnt[-1] == 0
        out[ang] = (F.min(), steps[np.flatnonzero(cnt > 0).max()], cnt[0])
    Fs = np.array([v[0] for v in out.values()])
    ds = np.array([v[1] for v in out.values()])
    A0 = np.array([v[2] for v in out.values()], dtype=float)
    assert Fs.max() < 0
    assert np.ptp(Fs) <= 0.05 * abs(Fs.mean())
    assert np.ptp(ds) <= 0.05 * abs(ds.mean())
    assert np.ptp(A0) <= 0.02 * A0.mean()
    assert abs(A0.mean() / n ** 2 - side ** 2) <= 0.02 * side ** 2
