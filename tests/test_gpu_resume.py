"""Checkpoint and resume of a sweep: the state a sweep ends in (its final
pressure and, when adhesive, the held contact set) is all a fresh handle needs
to continue, and a sweep split into two calls gives the single call's results
bitwise."""
import numpy as np
import pytest

from paper_1612_08395_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FIELDS = ("force", "area", "contact_radius", "final_eps", "max_gap_violation", "depth",
          "iterations", "detach_rounds", "contact_count", "status")


def same(a, b):
    for ra, rb in zip(a, b):
        for f in FIELDS:
            x, y = getattr(ra, f), getattr(rb, f)
            assert x == y or (np.isnan(x) and np.isnan(y)), f


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_refine"])
@pytest.mark.parametrize("adhesive", [True, False])
def test_split_sweep_equals_single_sweep(bem_mod, cuda_ok, prec, adhesive):
    n, k, nu = 64, 0.5, 0.3
    dx = 1.0 / n
    prof = I.paraboloid(n)
    if adhesive:
        gam, steps, cut = 1e-3, np.linspace(0.01, -0.03, 41), 17
    else:
        gam, steps, cut = 0.0, np.linspace(0.002, 0.02, 20), 7
    p_full = np.empty((n, n))
    with bem_mod.Handle(n, n, dx, dx, k, nu) as h:
        r_full, _ = h.sweep(prof, steps, dgamma=gam, final_pressure=p_full, precision=prec)
    p1 = np.empty((n, n))
    with bem_mod.Handle(n, n, dx, dx, k, nu) as h:
        r1, _ = h.sweep(prof, steps[:cut], dgamma=gam, final_pressure=p1, precision=prec)
        S1 = h.contact_set()
    assert S1.dtype == np.uint8 and S1.shape == (n, n)
    if adhesive:
        assert S1.sum() == r1[-1].contact_count
    p2 = np.empty((n, n))
    with bem_mod.Handle(n, n, dx, dx, k, nu) as h2:  # only the saved state carries over
        r2, _ = h2.sweep_from(prof, steps[cut:], p1, S1 if adhesive else None, dgamma=gam,
                              final_pressure=p2, precision=prec)
    same(r_full[:cut], r1)
    same(r_full[cut:], r2)
    assert np.array_equal(p_full, p2)


def test_adhesive_resume_needs_the_contact_set(bem_mod, cuda_ok):
    n = 32
    with bem_mod.Handle(n, n, 1.0 / n, 1.0 / n, 0.3, 0.3) as h:
        with pytest.raises(bem_mod.BemError) as e:
            h.sweep_from(I.paraboloid(n), [0.01, 0.0], np.zeros((n, n)), None, dgamma=1e-3)
    assert e.value.code == bem_mod.BEM_EINVAL
