"""Planted mistakes in the oracle, each caught by a pin.

Each test rewrites one line of an oracle function (in memory, on the CPU),
then runs a pin from test_oracle_pins.py's families against the mutant and
checks that the pin now fails.  This shows the pins would catch that kind of
error in the real oracle.  The oracle files on disk are never modified.
"""
import inspect
import textwrap

import numpy as np
import pytest

from paper_1612_08395_gb300 import inputs as I


def _mutant(func, old, new):
    src = textwrap.dedent(inspect.getsource(func))
    assert old in src, f"mutation anchor not found: {old!r}"
    ns = dict(func.__globals__)
    exec(compile(src.replace(old, new, 1), f"<mutant {func.__name__}>", "exec"), ns)
    return ns[func.__name__]


def _hertz_force_rel_error(oracle_mod, compliance):
    from oracle import closed_forms as CF
    n, k, nu, d = 32, 0.5, 0.3, 0.01
    dx = 1.0 / n
    A = compliance(k, nu)
    conv = oracle_mod.FFTConvolver(oracle_mod.influence_quarter(k, dx, dx, n + 1, n + 1), n, n)
    res = oracle_mod.pk_solve(A, conv, I.paraboloid(n), d)
    F = dx * dx * res.p.sum()
    return abs(F / CF.hertz_force(CF.hertz_radius(d, k, 1.0), k, nu, 1.0) - 1)


def test_dropped_poisson_factor_is_caught(oracle_mod):
    assert _hertz_force_rel_error(oracle_mod, oracle_mod.compliance) < 0.02
    bad = _mutant(oracle_mod.compliance, "(1.0 - nu * nu)", "1.0")
    assert _hertz_force_rel_error(oracle_mod, bad) > 0.05


def test_transposed_kernel_is_caught(oracle_mod):
    # Non-square cells (dy = 2 dx): building the torus from the transposed table
    # breaks FFT-equals-direct.
    n = 12
    Kq = oracle_mod.influence_quarter(-0.4, 1.0 / n, 2.0 / n, n + 1, n + 1)
    p = I.random_pressure(n, n, seed=4)
    ud = oracle_mod.convolve_direct(Kq[:n, :n], p)
    bad_torus = _mutant(oracle_mod.torus_kernel, "Kq[np.ix_(iy, ix)]", "Kq.T[np.ix_(iy, ix)]")

    def fft_conv(torus):
        return np.fft.irfft2(np.fft.rfft2(np.pad(p, ((0, n), (0, n))))
                             * np.fft.rfft2(torus(Kq, 2 * n, 2 * n)), s=(2 * n, 2 * n))[:n, :n]

    assert np.abs(fft_conv(oracle_mod.torus_kernel) - ud).max() < 1e-12 * np.abs(ud).max()
    assert np.abs(fft_conv(bad_torus) - ud).max() > 1e-3 * np.abs(ud).max()


def test_overlap_sign_is_caught(oracle_mod):
    import itertools
    n, k, nu = 3, 0.3, 0.3
    dx = 1.0 / n
    A = oracle_mod.compliance(k, nu)
    Kq = oracle_mod.influence_quarter(k, dx, dx, n + 1, n + 1)
    rng = np.random.Generator(np.random.PCG64(1))
    h = rng.random((n, n)) * 0.01
    d = 0.006
    Kfull = np.array([[Kq[abs(a // n - b // n), abs(a % n - b % n)] for b in range(n * n)]
                      for a in range(n * n)])
    ref = None
    for mask in itertools.product([False, True], repeat=n * n):
        S = np.array(mask)
        p = np.zeros(n * n)
        if S.any():
            p[S] = np.linalg.solve(A * Kfull[np.ix_(S, S)], (d - h.ravel())[S])
        g = A * Kfull @ p + h.ravel() - d
        if (p >= -1e-14).all() and (g[~S] >= -1e-14).all():
            ref = p
    bad = _mutant(oracle_mod.pk_solve, "p = np.where(Iol, -tau * g, p)",
                  "p = np.where(Iol, tau * g, p)")
    conv = oracle_mod.DirectConvolver(Kq, n, n)
    # start from one loaded element so that the overlap step has to bring in the rest
    p0 = np.zeros((n, n))
    p0[1, 1] = 1e-3
    good = oracle_mod.pk_solve(A, conv, h, d, p0=p0, tol=1e-14).p.ravel()
    assert np.allclose(good, ref, rtol=1e-9, atol=1e-12)
    res = bad(A, conv, h, d, p0=p0, tol=1e-14, max_iter=300)
    assert not np.allclose(res.p.ravel(), ref, rtol=1e-6, atol=1e-9)


def test_detach_sign_is_caught(oracle_mod):
    from oracle import closed_forms as CF
    n, k, nu, a, gam = 32, 0.0, 0.3, 0.2, 1e-3
    dx = 1.0 / n
    A = oracle_mod.compliance(k, nu)
    conv = oracle_mod.FFTConvolver(oracle_mod.influence_quarter(k, dx, dx, n + 1, n + 1), n, n)
    dc = CF.flat_punch_dcrit(a, k, nu, gam)
    steps = np.linspace(0.0, -1.3 * dc, 66)[1:]
    pc = oracle_mod.p_crit(k, nu, gam, dx)
    bad = _mutant(oracle_mod.adhesive_unload, "D = S & (-p > pcrit)", "D = S & (p > pcrit)")
    for fn, ok in ((oracle_mod.adhesive_unload, True), (bad, False)):
        out, _, _ = fn(A, conv, I.flat_punch(n, a), 0.2 * dc, steps, pc, dx * dx)
        lost = [o["d"] for o in out if o["count"] == 0]
        caught = bool(lost) and abs(lost[0] / -dc - 1) < 0.1
        assert caught == ok


@pytest.mark.parametrize("old,new", [("(2.0 ** k)", "(2.0 ** (-k))"),
                                     ("math.gamma(1.0 + k / 2.0)", "math.gamma(1.0 + k)"),
                                     ("math.gamma((3.0 + k - b) / 2.0)", "math.gamma((3.0 - k - b) / 2.0)")])
def test_alpha_mistakes_invisible_at_k0_are_caught(oracle_mod, old, new):
    # each mistake leaves alpha(0, nu) = 1/pi (the Boussinesq pin passes) but
    # breaks Gibson's limit alpha(k, 0.5) / (1 - k) -> 1/pi as k -> 1
    import math
    bad = _mutant(oracle_mod.alpha, old, new)
    k = 0.999

    def gibson_gap(f):
        return abs(math.pi * f(k, 0.5) / (1.0 - k) - 1.0)

    assert bad(0.0, 0.3) == pytest.approx(1.0 / math.pi, rel=1e-15)
    assert gibson_gap(oracle_mod.alpha) <= 1.0 - k
    assert gibson_gap(bad) > 10 * (1.0 - k)  # the pin (gap <= 1 - k) fails by a margin


def test_alpha_mistakes_split_between_the_two_pins(oracle_mod):
    # a dropped beta factor is invisible where beta = 1 (the Frohlich-Holl line)
    # but breaks Gibson's limit (beta -> 0); a wrong Gamma(2+k) keeps the
    # Boussinesq value at k = 0 and leaves the Frohlich-Holl line
    import math
    k = 0.999
    fh = lambda f, kk: f(kk, 1.0 / (2.0 + kk)) / ((2.0 + kk) / (2.0 * math.pi * (1.0 + kk) ** 2)) - 1.0
    no_beta = _mutant(oracle_mod.alpha, "(2.0 ** k) * b * math.sin", "(2.0 ** k) * math.sin")
    assert abs(fh(no_beta, 0.5)) < 1e-13
    assert abs(math.pi * no_beta(k, 0.5) / (1.0 - k) - 1.0) > 10 * (1.0 - k)
    bad_gamma = _mutant(oracle_mod.alpha, "math.gamma(2.0 + k)", "math.gamma(1.0 + k)")
    assert bad_gamma(0.0, 0.3) == pytest.approx(1.0 / math.pi, rel=1e-15)
    assert abs(fh(bad_gamma, 0.5)) > 0.1


def test_p_crit_element_size_exponent_is_caught(oracle_mod):
    # Eq. 24 scales with delta^-(1-k)/2; a flipped exponent breaks the energy
    # balance U_el = dgamma delta^2 (Eqs. 21-22) behind it
    k, nu, g, dl, c1 = 0.3, 0.3, 1e-3, 1.0 / 2048, 5.62
    A = oracle_mod.compliance(k, nu)

    def balance(f):
        pc = f(k, nu, g, dl, c1=c1)
        return A * pc ** 2 / 2 * dl ** (3 - k) * c1 / (g * dl * dl) - 1.0

    bad = _mutant(oracle_mod.p_crit, "delta ** (1.0 - k)", "delta ** (1.0 + k)")
    assert abs(balance(oracle_mod.p_crit)) < 1e-13
    assert abs(balance(bad)) > 0.5


def test_unmasked_fixed_set_transform_is_caught(oracle_mod):
    # the fixed-set CG must restrict r = A K t to the held set; without the mask
    # the iterate leaves the set and no longer solves the reduced system
    n, k = 6, -0.2
    dx = 1.0 / n
    A = oracle_mod.compliance(k, 0.3)
    Kq = oracle_mod.influence_quarter(k, dx, dx, n, n)
    conv = oracle_mod.DirectConvolver(Kq, n, n)
    rng = np.random.Generator(np.random.PCG64(5))
    S = rng.random((n, n)) < 0.6
    c = rng.random((n, n)) - 0.5
    Kfull = np.array([[Kq[abs(a // n - b // n), abs(a % n - b % n)] for b in range(n * n)]
                      for a in range(n * n)])
    s = S.ravel()
    ref = np.linalg.solve(A * Kfull[np.ix_(s, s)], -c.ravel()[s])
    bad = _mutant(oracle_mod.fixed_set_cg, "r = np.where(S, A * conv(t), 0.0)", "r = A * conv(t)")
    for fn, ok in ((oracle_mod.fixed_set_cg, True), (bad, False)):
        p = fn(A, conv, c, S, np.zeros((n, n)), tol=1e-14, max_iter=500).p.ravel()
        good = np.allclose(p[s], ref, rtol=1e-10, atol=1e-13) and np.all(p[~s] == 0)
        assert good == ok


def test_alpha_in_the_hertz_numerator_is_caught(oracle_mod):
    # reading R6: alpha divides Eq. 16; printed in the numerator, the closed form
    # no longer matches the BEM force of the same graded Hertz contact
    from oracle import closed_forms as CF
    bad = _mutant(CF.hertz_force, "4.0 * E0 * a ** (3.0 + k) / (alpha(k, nu) * gamma_pair(k)",
                  "4.0 * E0 * alpha(k, nu) * a ** (3.0 + k) / (gamma_pair(k)")
    n, k, nu, d = 32, 0.5, 0.3, 0.01
    dx = 1.0 / n
    A = oracle_mod.compliance(k, nu)
    conv = oracle_mod.FFTConvolver(oracle_mod.influence_quarter(k, dx, dx, n + 1, n + 1), n, n)
    F = dx * dx * oracle_mod.pk_solve(A, conv, I.paraboloid(n), d).p.sum()
    a = CF.hertz_radius(d, k, 1.0)
    assert abs(F / CF.hertz_force(a, k, nu, 1.0) - 1) < 0.02
    assert abs(F / bad(a, k, nu, 1.0) - 1) > 0.5
