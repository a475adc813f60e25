"""Fixed-set solves on the contact set only (adhesive algorithm, Sec. 3.1).

The fixed-set CG runs on the rows of the contact set and on the smallest
torus that holds the contact box; these cases put the box where that is
delicate: against the grid's corner (the sub-grid runs past the grid edge),
on a rectangular grid (different torus sizes in x and y), and with a box that
shrinks across torus sizes during the unloading.  Each is compared step by
step with the FP64 oracle, which always solves on the whole grid.
"""
import numpy as np
import pytest

from paper_1612_08395_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def relL2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def shifted_paraboloid(nx, ny, dx, cx, cy, R=1.0):
    """h = ((x - cx)^2 + (y - cy)^2) / 2R on the element centres."""
    x = I.centres(nx, dx)
    y = I.centres(ny, dx)
    X, Y = np.meshgrid(x, y)
    return np.ascontiguousarray(((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * R))


def run_case(bem_mod, oracle_mod, nx, ny, k, nu, gam, d0, d_end, nsteps, cx, cy, prec):
    dx = 1.0 / nx
    prof = shifted_paraboloid(nx, ny, dx, cx, cy)
    A = oracle_mod.compliance(k, nu)
    conv = oracle_mod.DirectConvolver(oracle_mod.influence_quarter(k, dx, dx, nx, ny), ny, nx)
    steps = np.linspace(d0, d_end, nsteps)
    out, p_ref, _ = oracle_mod.adhesive_unload(A, conv, prof, d0, steps[1:],
                                               oracle_mod.p_crit(k, nu, gam, dx), dx * dx,
                                               tol_pk=1e-12, tol_cg=1e-13)
    p = np.empty((ny, nx))
    with bem_mod.Handle(nx, ny, dx, dx, k, nu) as h:
        res, rc = h.sweep(prof, steps, dgamma=gam, final_pressure=p, precision=prec, tol=1e-12)
    assert rc == bem_mod.BEM_OK
    assert sum(o["count"] for o in out) > 0
    for o, r in zip(out, res[1:]):
        assert r.contact_count == o["count"], (o["d"], r.contact_count, o["count"])
        assert r.force == pytest.approx(o["force"], rel=1e-8, abs=1e-14)
    assert relL2(p, p_ref) <= 1e-9 or (p_ref == 0).all() and (p == 0).all()


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_contact_box_at_grid_corner(bem_mod, oracle_mod, cuda_ok, prec):
    # contact centred 4 elements from the top right corner: the sub-grid placed at
    # the box origin extends past both grid edges
    n = 64
    c = 0.5 - 4.5 / n
    run_case(bem_mod, oracle_mod, n, n, 0.5, 0.3, 1e-3, 0.01, -0.03, 31, c, c, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_contact_box_rectangular_grid(bem_mod, oracle_mod, cuda_ok, prec):
    # 80 x 48 square elements: tori 256 x 128; the contact sits off centre
    run_case(bem_mod, oracle_mod, 80, 48, -0.3, 0.3, 2e-3, 0.006, -0.02, 25, -0.12, 0.05, prec)


def test_contact_box_shrinks_across_tori(bem_mod, oracle_mod, cuda_ok):
    # a wide preload whose box needs half the torus (no smaller torus at first),
    # then shrinks through smaller ones while unloading
    run_case(bem_mod, oracle_mod, 64, 64, 0.0, 0.3, 5e-4, 0.09, -0.03, 41, 0.0, 0.0, "fp64")
