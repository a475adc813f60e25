"""Fixed-set solves on the contact set only (adhesive algorithm, Sec. 3.1), and
the host-side fault injection around them (sub-context allocation failure,
forced iteration cap).

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


INJECT = r"""
import json, sys
import numpy as np
sys.path.insert(0, %r)
import paper_1612_08395_gb300.bem as bem
import paper_1612_08395_gb300.inputs as I
n = 128
prof = I.paraboloid(n)
p = np.empty((n, n))
q = np.empty((n, n))
with bem.Handle(n, n, 1.0 / n, 1.0 / n, 0.3, 0.3) as h:
    res, rc = h.sweep(prof, np.linspace(0.004, -0.01, 29), dgamma=1e-3, final_pressure=p,
                      precision="fp64", tol=1e-12)
    r1, rc1 = h.solve(prof, 0.002, pressure_out=q, precision="fp32_refine")
    b1 = h.info().device_bytes
np.save(sys.argv[1], np.stack([p, q]))
print(json.dumps({"rc": [rc, rc1], "F": [r.force for r in res] + [r1.force],
                  "cnt": [r.contact_count for r in res] + [r1.contact_count], "bytes": b1}))
"""


def test_sub_context_failure_falls_back_to_whole_grid(tmp_path, cuda_ok):
    """Host-side fault injection: with every contact-box sub-context creation
    failing (as an allocation failure would), solves run on the whole grid and
    give the same results."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = {}
    for inj in ("0", "1"):
        f = str(tmp_path / f"p{inj}.npy")
        env = dict(os.environ, BEM_INJECT_SUB_FAILURE=inj)
        r = subprocess.run([sys.executable, "-c", INJECT % root, f], capture_output=True, text=True,
                           env=env, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        out[inj] = (json.loads(r.stdout.strip().splitlines()[-1]), np.load(f))
    (a, pa), (b, pb) = out["0"], out["1"]
    assert a["rc"] == [0, 0] and b["rc"] == [0, 0]
    assert a["bytes"] > b["bytes"]  # sub-contexts were made only without the injection
    assert a["cnt"] == b["cnt"]
    np.testing.assert_allclose(b["F"], a["F"], rtol=1e-9, atol=1e-15)
    assert relL2(pb[0], pa[0]) <= 1e-10 or (pa[0] == 0).all() and (pb[0] == 0).all()
    assert relL2(pb[1], pa[1]) <= 1e-9


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_forced_iteration_cap_reports_noconv(bem_mod, cuda_ok, prec):
    """An iteration cap below what the tolerance needs ends the solve with
    BEM_ENOCONV, the result filled from the last iterate."""
    n = 128
    p = np.empty((n, n))
    with bem_mod.Handle(n, n, 1.0 / n, 1.0 / n, 0.5, 0.3) as h:
        res, rc = h.solve(I.paraboloid(n), 0.01, pressure_out=p, precision=prec, tol=1e-14, max_iter=5)
    assert rc == bem_mod.BEM_ENOCONV and res.status == bem_mod.BEM_ENOCONV
    assert res.iterations == 5
    assert np.isfinite(p).all() and p.min() >= 0.0 and res.contact_count == int((p > 0).sum())
    assert res.force == pytest.approx(p.sum() / n / n, rel=1e-12)
