"""Pins of the FP64 oracle against what the paper and the mathematics fix.

No GPU.  Each test names the passage or identity it checks.  Together they
are meant to catch a dropped term, a wrong sign or index, or a transposed
operand anywhere in the oracle (see test_oracle_mutations.py for planted
mistakes that these pins catch).
"""
import itertools
import math

import numpy as np
import pytest
from scipy import integrate

from conftest import read_golden
from paper_1612_08395_gb300 import inputs as I


# ---------------------------------------------------------------- Eqs. 3-4
@pytest.mark.parametrize("nu", [0.0, 0.25, 0.3, 0.45, 0.5])
def test_alpha_homogeneous_is_boussinesq(oracle_mod, nu):
    # k = 0: Eq. 2 must reduce to Boussinesq's u = (1-nu^2) F / (pi E r).
    assert oracle_mod.alpha(0.0, nu) == pytest.approx(1.0 / math.pi, rel=1e-15)
    assert oracle_mod.beta(0.0, nu) == pytest.approx(1.0, rel=1e-15)


@pytest.mark.parametrize("k", [0.99, 0.999, 0.9999])
def test_alpha_gibson_limit(oracle_mod, k):
    # k -> 1 at nu = 0.5 is Gibson's incompressible soil (shear modulus m z, so
    # E0 / c0 = 3 m): its surface responds locally, w = p / (2 m) (Gibson 1967).
    # The kernel (1 - k) / (2 pi r^(1+k)) tends to the 2D delta, so Eq. 2 gives
    # w -> alpha (1 - nu^2) c0 p 2 pi / ((1 - k) E0) and alpha / (1 - k) -> 1 / pi,
    # independently of Eq. 3; the approach is linear in 1 - k.
    ratio = math.pi * oracle_mod.alpha(k, 0.5) / (1.0 - k)
    assert abs(ratio - 1.0) <= 1.0 - k


@pytest.mark.parametrize("k", [0.05, 0.2, 0.3, 0.5, 0.7, 0.9])
def test_alpha_frohlich_holl(oracle_mod, k):
    # nu = 1/(2+k) (beta = 1): the point-load field of E = E0 (z/c0)^k is purely
    # radial, sigma_R = n F cos^(n-2)(theta) / (2 pi R^2) with n = 3 + k (it carries F
    # and satisfies equilibrium).  Integrating its strains sigma_R/E and -nu sigma_R/E
    # in spherical coordinates gives u_R ~ cos(theta) / R^(1+k) and u_theta ~
    # sin(theta) / R^(1+k) with zero shear strain, and at the surface
    # |u_z| = n F c0^k / (2 pi (1+k) (2+k) E0 r^(1+k)).  Matching Eq. 2 with
    # 1 - nu^2 = (1+k)(3+k)/(2+k)^2 gives alpha = (2+k) / (2 pi (1+k)^2).
    nu = 1.0 / (2.0 + k)
    assert oracle_mod.beta(k, nu) == pytest.approx(1.0, rel=1e-14)
    assert oracle_mod.alpha(k, nu) == pytest.approx((2.0 + k) / (2.0 * math.pi * (1.0 + k) ** 2),
                                                     rel=1e-13)


def test_beta_definition(oracle_mod):
    # Eq. 4 at nu = 0 is sqrt(1+k); at nu = 0.5 it is sqrt((1+k)(1-k)).
    for k in (-0.7, -0.2, 0.4, 0.9):
        assert oracle_mod.beta(k, 0.0) == pytest.approx(math.sqrt(1 + k), rel=1e-15)
        assert oracle_mod.beta(k, 0.5) == pytest.approx(math.sqrt((1 + k) * (1 - k)), rel=1e-15)


# ---------------------------------------------------------------- Eq. 9
@pytest.mark.parametrize("di,dj", [(0, 0), (1, 0), (0, 2), (1, 1), (3, 2), (7, 0), (9, 5)])
@pytest.mark.parametrize("dx,dy", [(1.0, 1.0), (0.37, 0.37), (1 / 64, 1 / 128)])
def test_K_equals_love_at_k0(oracle_mod, di, dj, dx, dy):
    # k = 0 is the homogeneous medium: Love's closed form for a uniformly loaded rectangle.
    from oracle.closed_forms import love_rect
    a0, a1 = (di - 0.5) * dx, (di + 0.5) * dx
    b0, b1 = (dj - 0.5) * dy, (dj + 0.5) * dy
    v = oracle_mod.influence_rect(0.0, a0, a1, b0, b1)
    assert v == pytest.approx(love_rect(a0, a1, b0, b1), rel=1e-12)


@pytest.mark.parametrize("k", [-0.9, -0.5, -0.2, 0.3, 0.7, 0.9])
@pytest.mark.parametrize("di,dj", [(1, 1), (2, 3), (5, 1), (4, 4)])
def test_K_equals_eq11_off_axis(oracle_mod, k, di, dj):
    # Eq. 11 (hypergeometric closed form) holds when the element does not straddle
    # the observation row or column.
    from oracle.closed_forms import eq11
    q, p = di - 0.5, di + 0.5
    n, m = dj - 0.5, dj + 0.5
    v = oracle_mod.influence_rect(k, q, p, n, m)
    assert v == pytest.approx(eq11(k, q, p, n, m), rel=1e-11)


@pytest.mark.parametrize("k", [-0.8, 0.0, 0.6])
def test_K_homogeneity(oracle_mod, k):
    # Eq. 9 scales as K(lambda dx) = lambda^(1-k) K(dx) (degree 2 - (1+k)).
    K1 = oracle_mod.influence_quarter(k, 1.0, 1.0, 6, 5)
    Kl = oracle_mod.influence_quarter(k, 0.125, 0.125, 6, 5)
    np.testing.assert_allclose(Kl, 0.125 ** (1 - k) * K1, rtol=1e-12)


@pytest.mark.parametrize("k", [-0.9, -0.3, 0.5, 0.9])
def test_K_far_field(oracle_mod, k):
    # Far from the element, K -> dx dy / r^(1+k) with a relative error O((dx/r)^2).
    dx = 0.5
    for n in (10, 40, 160):
        v = oracle_mod.influence_rect(k, (n - 0.5) * dx, (n + 0.5) * dx, 2.5 * dx, 3.5 * dx)
        r = dx * math.hypot(n, 3)
        rel = v / (dx * dx * r ** (-(1 + k))) - 1
        assert abs(rel) < 0.2 / (n * n + 9)


def test_K_nonsquare_transpose(oracle_mod):
    # Swapping the element sides swaps the offsets: K_{dx,dy}(di,dj) = K_{dy,dx}(dj,di).
    Ka = oracle_mod.influence_quarter(0.4, 0.02, 0.05, 7, 5)
    Kb = oracle_mod.influence_quarter(0.4, 0.05, 0.02, 5, 7)
    np.testing.assert_allclose(Ka, Kb.T, rtol=1e-13)


@pytest.mark.parametrize("k", [-0.9, -0.5, 0.0, 0.5, 0.9])
def test_spectrum_positive(oracle_mod, k):
    # K is symmetric positive definite: its spectrum on the even-extended torus is > 0.
    n = 32
    Kq = oracle_mod.influence_quarter(k, 1.0 / n, 1.0 / n, n + 1, n + 1)
    conv = oracle_mod.FFTConvolver(Kq, n, n)
    assert np.abs(conv.khat.imag).max() < 1e-12 * np.abs(conv.khat.real).max()
    assert conv.khat.real.min() > 0


# ---------------------------------------------------------------- Eq. 23, Table 1
def test_c1_k0_closed_form(oracle_mod):
    from oracle.closed_forms import c1_k0_exact
    assert oracle_mod.c1_uncorrected(0.0) == pytest.approx(c1_k0_exact(), rel=1e-12)


def test_c1_k0_agrees_with_table1(oracle_mod):
    # Table 1 lists the corrected c1(0) = 2.97; the uncorrected integral is 2.97321.
    assert round(oracle_mod.c1_uncorrected(0.0), 2) == 2.97


def test_c1_uncorrected_by_plain_quadrature(oracle_mod):
    # The reduced 2D form agrees with scipy's adaptive quadrature of the same integral.
    for k in (-0.6, 0.5):
        f = lambda v, u: 4 * (1 - u) * (1 - v) * (u * u + v * v) ** (-(1 + k) / 2)
        ref, _ = integrate.dblquad(f, 0, 1, 0, 1, epsabs=1e-13, epsrel=1e-11)
        assert oracle_mod.c1_uncorrected(k) == pytest.approx(ref, rel=1e-8)


def test_table1_matches_paper_fixture(oracle_mod):
    rows = sorted(read_golden("table1_c1.txt"))
    np.testing.assert_array_equal(oracle_mod.TABLE1_K, [r[0] for r in rows])
    np.testing.assert_array_equal(oracle_mod.TABLE1_C1, [r[1] for r in rows])


def test_c1_spline_reproduces_table(oracle_mod):
    for k, c in zip(oracle_mod.TABLE1_K, oracle_mod.TABLE1_C1):
        assert oracle_mod.c1_corrected(float(k)) == pytest.approx(c, rel=1e-13)
    ks = np.linspace(-0.9, 0.9, 181)
    vals = [oracle_mod.c1_corrected(float(k)) for k in ks]
    assert np.all(np.diff(vals) > 0)  # monotone like the table


def test_p_crit_eq24(oracle_mod):
    # Eq. 24 from U_el = U_surf with Eqs. 21 (p^2) and 22.
    k, nu, g, dl = 0.3, 0.3, 1e-3, 1.0 / 2048
    pc = oracle_mod.p_crit(k, nu, g, dl)
    A = oracle_mod.compliance(k, nu)
    u_el = A * pc ** 2 / 2 * dl ** (3 - k) * 5.62
    assert u_el == pytest.approx(g * dl * dl, rel=1e-13)


# ---------------------------------------------------------------- Eq. 7 vs Eq. 13
@pytest.mark.parametrize("ny,nx", [(4, 4), (7, 7), (16, 16), (9, 20), (33, 17)])
@pytest.mark.parametrize("workers", [1, 4])
def test_fft_equals_direct(oracle_mod, ny, nx, workers):
    k = -0.4
    Kq = oracle_mod.influence_quarter(k, 1.0 / nx, 1.0 / ny, nx + 1, ny + 1)
    p = I.random_pressure(nx, ny, seed=3)
    ud = oracle_mod.convolve_direct(Kq[:ny, :nx], p)
    uf = oracle_mod.FFTConvolver(Kq, ny, nx, workers=workers)(p)
    assert np.abs(ud - uf).max() <= 1e-12 * np.abs(ud).max()


def test_direct_sum_by_hand(oracle_mod):
    # Tiny case written out: u_00 = sum_j K(|0-jx|, |0-jy|) p_j.
    Kq = oracle_mod.influence_quarter(0.2, 0.1, 0.1, 3, 2)
    p = np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 6.0]])
    u = oracle_mod.convolve_direct(Kq, p)
    hand = sum(Kq[abs(0 - jy), abs(1 - jx)] * p[jy, jx] for jy in range(2) for jx in range(3))
    assert u[0, 1] == pytest.approx(hand, rel=1e-15)
    at = oracle_mod.convolve_direct_at(Kq, p, np.array([1, 5]))
    np.testing.assert_allclose(at, u.ravel()[[1, 5]], rtol=1e-15)


# ---------------------------------------------------------------- the inverse problem
def _brute_force_lcp(A, Kfull, h, d):
    """Unique solution of the LCP by trying every contact set (tiny grids only)."""
    n = len(h)
    sols = []
    for mask in itertools.product([False, True], repeat=n):
        S = np.array(mask)
        p = np.zeros(n)
        if S.any():
            p[S] = np.linalg.solve(A * Kfull[np.ix_(S, S)], (d - h)[S])
        g = A * Kfull @ p + h - d
        if (p >= -1e-14).all() and (g[~S] >= -1e-14).all():
            sols.append(p)
    return sols


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pk_equals_brute_force_lcp(oracle_mod, seed):
    # The discrete non-adhesive problem is a strictly convex LCP with one solution;
    # enumerate all 2^9 contact sets of a 3x3 grid and compare.
    n, k, nu = 3, 0.3, 0.3
    dx = 1.0 / n
    A = oracle_mod.compliance(k, nu)
    Kq = oracle_mod.influence_quarter(k, dx, dx, n + 1, n + 1)
    rng = np.random.Generator(np.random.PCG64(seed))
    h = rng.random((n, n)) * 0.01
    d = 0.006
    Kfull = np.array([[Kq[abs(a // n - b // n), abs(a % n - b % n)] for b in range(n * n)]
                      for a in range(n * n)])
    sols = _brute_force_lcp(A, Kfull, h.ravel(), d)
    assert len(sols) == 1
    res = oracle_mod.pk_solve(A, oracle_mod.DirectConvolver(Kq, n, n), h, d, tol=1e-14)
    np.testing.assert_allclose(res.p.ravel(), sols[0], rtol=1e-9, atol=1e-12)


@pytest.fixture(scope="module")
def config1(oracle_mod):
    """64 x 64, k = 0.5, nu = 0.3, paraboloid R = 1, d = 0.01, tol 1e-10."""
    n, k, nu, d, R = 64, 0.5, 0.3, 0.01, 1.0
    dx = 1.0 / n
    A = oracle_mod.compliance(k, nu)
    Kq = oracle_mod.influence_quarter(k, dx, dx, n + 1, n + 1)
    h = I.paraboloid(n, R)
    res = oracle_mod.pk_solve(A, oracle_mod.DirectConvolver(Kq, n, n), h, d, tol=1e-10)
    return dict(n=n, k=k, nu=nu, d=d, R=R, dx=dx, A=A, Kq=Kq, h=h, res=res)


def test_config1_graded_hertz(oracle_mod, config1):
    from oracle import closed_forms as CF
    c = config1
    res = c["res"]
    assert res.converged
    a = CF.hertz_radius(c["d"], c["k"], c["R"])
    F = c["dx"] ** 2 * res.p.sum()
    assert F == pytest.approx(CF.hertz_force(a, c["k"], c["nu"], c["R"]), rel=5e-3)
    # area within one ring of elements of pi a^2
    area = c["dx"] ** 2 * (res.p > 0).sum()
    assert abs(area - math.pi * a * a) <= 2 * math.pi * a * c["dx"]


def test_config1_complementarity(oracle_mod, config1):
    res = config1["res"]
    d = config1["d"]
    Ic = res.p > 0
    assert res.p.min() >= 0
    assert np.abs(res.g[Ic]).max() < 1e-9 * d
    assert res.g[~Ic].min() > -1e-9 * d


def test_config1_d4_symmetry(oracle_mod, config1):
    # Centred axisymmetric indenter: p is symmetric under the grid's symmetries (Fig. 9).
    p = config1["res"].p
    scale = p.max()
    for q in (p[::-1, :], p[:, ::-1], p.T):
        assert np.abs(q - p).max() < 1e-8 * scale


def test_config1_deflection_eq14(oracle_mod, config1):
    # Surface deflection d - h inside and A K p outside against Eq. 14.
    from oracle import closed_forms as CF
    c = config1
    u = c["A"] * oracle_mod.convolve_direct(c["Kq"][:c["n"], :c["n"]], c["res"].p)
    r = I.radius_grid(c["n"], c["n"], c["dx"])
    a = CF.hertz_radius(c["d"], c["k"], c["R"])
    sel = (r > 1.3 * a) & (r < 0.45)
    ref = CF.hertz_deflection(r[sel], a, c["k"], c["R"])
    assert np.abs(u[sel] - ref).max() < 0.02 * c["d"]
    # Eq. 14 at r = 0 is a^2 / ((1+k) R) = d (Eq. 15)
    assert CF.hertz_deflection(np.array([0.0]), a, c["k"], c["R"])[0] == pytest.approx(c["d"])


@pytest.mark.parametrize("k,n", [(0.5, 64), (-0.5, 128)])
def test_pressure_profiles_match_bem(oracle_mod, k, n):
    # The graded Hertz pressure 2 cos(pi k/2) (a^2 - r^2)^((1+k)/2) / ((1+k)^2 R pi^2 A)
    # and the flat-punch pressure p0 (1 - r^2/a^2)^(-(1-k)/2) against the BEM pressure
    # field, away from the contact edge where the discretisation smears the profile.
    from oracle import closed_forms as CF
    nu, d = 0.3, 0.01
    dx = 1.0 / n
    A = oracle_mod.compliance(k, nu)
    conv = oracle_mod.FFTConvolver(oracle_mod.influence_quarter(k, dx, dx, n + 1, n + 1), n, n)
    r = I.radius_grid(n, n, dx)
    p = oracle_mod.pk_solve(A, conv, I.paraboloid(n), d, tol=1e-10).p
    a = CF.hertz_radius(d, k, 1.0)
    ref = CF.hertz_pressure(r, a, k, nu, 1.0)
    sel = r < 0.7 * a
    assert np.abs(p[sel] - ref[sel]).max() <= 0.01 * ref.max()
    ap = 0.2
    p = oracle_mod.pk_solve(A, conv, I.flat_punch(n, ap), d, tol=1e-10).p
    ref = CF.flat_punch_pressure(r, ap, d, k, nu)
    sel = r < 0.5 * ap
    assert np.abs(p[sel] - ref[sel]).max() <= 0.03 * ref[sel].min()


def test_pressure_fields_integrate_to_forces(oracle_mod):
    from oracle import closed_forms as CF
    for k in (-0.6, 0.0, 0.4):
        a, nu, R, d = 0.15, 0.3, 1.0, 0.01
        F, _ = integrate.quad(lambda r: 2 * math.pi * r * CF.hertz_pressure(r, a, k, nu, R), 0, a,
                              limit=200)
        assert F == pytest.approx(CF.hertz_force(a, k, nu, R), rel=1e-7)
        Fp, _ = integrate.quad(lambda r: 2 * math.pi * r * CF.flat_punch_pressure(r, a, d, k, nu),
                               0, a, limit=200)
        assert Fp == pytest.approx(CF.flat_punch_stiffness(a, k, nu) * d, rel=1e-6)
    # k = 0: Hertz and Kendall
    Es = 1 / (1 - 0.3 ** 2)
    assert CF.hertz_force(0.1, 0.0, 0.3, 2.0) == pytest.approx(4 * Es * 0.1 ** 3 / (3 * 2.0))
    assert CF.flat_punch_fcrit(0.1, 0.0, 0.3, 1e-3) == pytest.approx(
        math.sqrt(8 * math.pi * 1e-3 * Es * 0.1 ** 3))
    for k in (-0.5, 0.3):
        S = CF.flat_punch_stiffness(0.2, k, 0.3)
        assert CF.flat_punch_fcrit(0.2, k, 0.3, 1e-3) == pytest.approx(
            S * CF.flat_punch_dcrit(0.2, k, 0.3, 1e-3), rel=1e-13)


def test_normalised_hertz_curve(oracle_mod):
    # Eq. 17 (alpha in the numerator) collapses Eq. 16 onto F~ = d~^((3+k)/2).
    from oracle import closed_forms as CF
    for k in (-0.8, 0.0, 0.8):
        d, R = 0.013, 1.7
        F = CF.hertz_force(CF.hertz_radius(d, k, R), k, 0.3, R)
        dn, Fn = CF.hertz_normalised(d, F, k, 0.3, R)
        assert Fn == pytest.approx(dn ** ((3 + k) / 2), rel=1e-12)


@pytest.mark.parametrize("k", [-0.5, 0.5])
def test_flat_punch_stiffness(oracle_mod, k):
    from oracle import closed_forms as CF
    n, nu, a, d = 64, 0.3, 0.2, 0.01
    dx = 1.0 / n
    A = oracle_mod.compliance(k, nu)
    Kq = oracle_mod.influence_quarter(k, dx, dx, n + 1, n + 1)
    res = oracle_mod.pk_solve(A, oracle_mod.FFTConvolver(Kq, n, n), I.flat_punch(n, a), d)
    F = dx * dx * res.p.sum()
    assert F == pytest.approx(CF.flat_punch_stiffness(a, k, nu) * d, rel=1e-2)


def test_monotone_force_depth(oracle_mod):
    n, k, nu = 32, -0.3, 0.3
    dx = 1.0 / n
    A = oracle_mod.compliance(k, nu)
    conv = oracle_mod.FFTConvolver(oracle_mod.influence_quarter(k, dx, dx, n + 1, n + 1), n, n)
    h = I.paraboloid(n)
    Fs, p = [], None
    for d in np.linspace(0.002, 0.02, 8):
        res = oracle_mod.pk_solve(A, conv, h, d, p0=p)
        p = res.p
        Fs.append(p.sum())
    assert np.all(np.diff(Fs) > 0)


def test_separated_indenter(oracle_mod):
    n = 8
    A = oracle_mod.compliance(0.2, 0.3)
    conv = oracle_mod.FFTConvolver(oracle_mod.influence_quarter(0.2, 1 / n, 1 / n, n + 1, n + 1), n, n)
    res = oracle_mod.pk_solve(A, conv, I.paraboloid(n) + 0.1, 0.05)
    assert res.p.sum() == 0.0 and res.converged


# ---------------------------------------------------------------- adhesion (Sec. 3)
def test_adhesive_flat_punch_eq25_eq26(oracle_mod):
    # Flat punch k = -0.5 (Fig. 6): detachment depth and force vs Eqs. 25-26.
    from oracle import closed_forms as CF
    n, k, nu, a, gam = 64, -0.5, 0.3, 0.2, 1e-3
    dx = 1.0 / n
    A = oracle_mod.compliance(k, nu)
    conv = oracle_mod.FFTConvolver(oracle_mod.influence_quarter(k, dx, dx, n + 1, n + 1), n, n)
    dc = CF.flat_punch_dcrit(a, k, nu, gam)
    Fc = CF.flat_punch_fcrit(a, k, nu, gam)
    steps = np.linspace(0.0, -1.3 * dc, 131)[1:]
    out, p, S = oracle_mod.adhesive_unload(A, conv, I.flat_punch(n, a), 0.2 * dc, steps,
                                           oracle_mod.p_crit(k, nu, gam, dx), dx * dx)
    last = [o for o in out if o["count"] > 0][-1]
    assert last["d"] / -dc == pytest.approx(1.0, abs=0.05)
    assert min(o["force"] for o in out) / -Fc == pytest.approx(1.0, abs=0.05)
    assert out[-1]["count"] == 0


def test_adhesive_paraboloid_jkr(oracle_mod):
    # Paraboloid k = 0.5 (Fig. 7): pull-off force vs the JKR-type closed form.
    from oracle import closed_forms as CF
    n, k, nu, R, gam, d0 = 64, 0.5, 0.3, 1.0, 1e-3, 0.01
    dx = 1.0 / n
    A = oracle_mod.compliance(k, nu)
    conv = oracle_mod.FFTConvolver(oracle_mod.influence_quarter(k, dx, dx, n + 1, n + 1), n, n)
    a0 = CF.hertz_radius(d0, k, R)
    aa = np.linspace(1e-3, a0, 4000)
    Fmin = min(CF.jkr_force(x, k, nu, R, gam) for x in aa)
    dmin = min(CF.jkr_depth(x, k, nu, R, gam) for x in aa)
    steps = np.arange(d0, 1.3 * dmin, -(d0 - dmin) / 150)[1:]
    out, p, S = oracle_mod.adhesive_unload(A, conv, I.paraboloid(n, R), d0, steps,
                                           oracle_mod.p_crit(k, nu, gam, dx), dx * dx)
    assert min(o["force"] for o in out) == pytest.approx(Fmin, rel=0.05)
    last = [o for o in out if o["count"] > 0][-1]
    assert last["d"] == pytest.approx(dmin, rel=0.08)
    # no element outside the contact area penetrates the indenter
    g = A * conv(p) + I.paraboloid(n, R) - steps[-1]
    assert g[~S].min() > -1e-12


def test_fixed_set_cg_solves_linear_system(oracle_mod):
    n, k = 6, -0.2
    dx = 1.0 / n
    A = oracle_mod.compliance(k, 0.3)
    Kq = oracle_mod.influence_quarter(k, dx, dx, n, n)
    conv = oracle_mod.DirectConvolver(Kq, n, n)
    rng = np.random.Generator(np.random.PCG64(5))
    S = rng.random((n, n)) < 0.6
    c = rng.random((n, n)) - 0.5
    res = oracle_mod.fixed_set_cg(A, conv, c, S, np.zeros((n, n)), tol=1e-14)
    Kfull = np.array([[Kq[abs(a // n - b // n), abs(a % n - b % n)] for b in range(n * n)]
                      for a in range(n * n)])
    s = S.ravel()
    ref = np.linalg.solve(A * Kfull[np.ix_(s, s)], -c.ravel()[s])
    np.testing.assert_allclose(res.p.ravel()[s], ref, rtol=1e-10, atol=1e-13)
    assert np.all(res.p.ravel()[~s] == 0)
