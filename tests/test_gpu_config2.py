"""All twelve warm-started 512 x 512 sweeps of the non-adhesive study: k in
{-0.5, 0, 0.5} x nu in {0.3, 0.5} x {paraboloid R = 1, flat punch of radius
0.2}, 50 depths d_j = 0.02 j / 50.

Per curve: the FP64 path against the oracle at the last depth; the FP32 path
with FP64 refinement against the FP64 path at every depth; forces against the
graded Hertz (Eqs. 15, 16) and flat-punch closed forms at every depth; and the
exact nu scaling of the discrete problem: nu enters only through the compliance
A of Eq. 12, so the solution for nu' is the one for nu times A(nu) / A(nu')."""
import numpy as np
import pytest

from paper_1612_08395_gb300 import inputs as I

pytestmark = pytest.mark.gpu

N = 512
DS = 0.02 * np.arange(1, 51) / 50


def relL2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("shape", ["paraboloid", "flat"])
@pytest.mark.parametrize("k", [-0.5, 0.0, 0.5])
def test_config2_curves(bem_mod, oracle_mod, cuda_ok, k, shape):
    from oracle import closed_forms as CF
    dx = 1.0 / N
    prof = I.paraboloid(N) if shape == "paraboloid" else I.flat_punch(N, 0.2)
    if shape == "paraboloid":
        closed = np.array([CF.hertz_force(CF.hertz_radius(d, k, 1.0), k, 0.3, 1.0) for d in DS])
        cf_tol = 1e-3
    else:
        closed = CF.flat_punch_stiffness(0.2, k, 0.3) * DS
        cf_tol = 2e-3
    out = {}
    for nu in (0.3, 0.5):
        A_ratio = oracle_mod.compliance(k, 0.3) / oracle_mod.compliance(k, nu)
        with bem_mod.Handle(N, N, dx, dx, k, nu) as h:
            for prec in ("fp64", "fp32_refine"):
                p = np.empty((N, N))
                res, rc = h.sweep(prof, DS, final_pressure=p, precision=prec,
                                  tol=1e-12 if prec == "fp64" else 0.0)
                assert rc == bem_mod.BEM_OK
                F = np.array([r.force for r in res])
                cnt = np.array([r.contact_count for r in res])
                out[nu, prec] = (F, cnt, p)
                # Eqs. 15-16 (paraboloid) and the flat-punch stiffness, scaled to nu
                np.testing.assert_allclose(F, closed * A_ratio, rtol=cf_tol)
        F64, c64, p64 = out[nu, "fp64"]
        F32, c32, p32 = out[nu, "fp32_refine"]
        np.testing.assert_allclose(F32, F64, rtol=1e-5)
        assert relL2(p32, p64) <= 1e-5
        assert np.all(np.abs(c32 - c64) <= np.maximum(2, 1e-3 * c64))
        if shape == "paraboloid":
            assert np.all(np.diff(F64) > 0) and np.all(np.diff(c64) >= 0)
        else:
            # the punch face is in full contact at every depth: F is linear in d
            assert np.all(c64 == c64[0])
            np.testing.assert_allclose(F64 / DS, F64[-1] / DS[-1], rtol=1e-9)
    # nu scaling of the discrete solution (unique: strictly convex problem)
    r = oracle_mod.compliance(k, 0.3) / oracle_mod.compliance(k, 0.5)
    assert relL2(out[0.5, "fp64"][2], out[0.3, "fp64"][2] * r) <= 1e-10
    assert np.array_equal(out[0.5, "fp64"][1], out[0.3, "fp64"][1])
    # the oracle (FFT mode, FP64) at the last depth
    A = oracle_mod.compliance(k, 0.3)
    conv = oracle_mod.FFTConvolver(oracle_mod.influence_quarter(k, dx, dx, N + 1, N + 1), N, N)
    ref = oracle_mod.pk_solve(A, conv, prof, DS[-1], tol=1e-12).p
    assert relL2(out[0.3, "fp64"][2], ref) <= 1e-10
    assert out[0.3, "fp64"][1][-1] == int((ref > 0).sum())
