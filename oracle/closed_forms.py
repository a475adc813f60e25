"""Closed-form solutions the oracle is pinned against (TEST INFRASTRUCTURE ONLY).

Each relation cites the equation it restates.  Two printed formulas carry a
misplaced alpha(k, nu) and are used in corrected form, with the reason:

  C1  Eq. 16 prints 4 alpha / (Gamma Gamma ...) E0/((1-nu^2) c0^k); the force
      must scale like 1/(alpha (1-nu^2) c0^k / E0), the compliance of Eq. 2,
      so alpha belongs in the denominator.  At k = 0 the corrected form is
      Hertz's F = 4 E* a^3 / (3 R) with E* = E0/(1-nu^2); integrating the
      pressure of ``hertz_pressure`` over the contact gives the same form.
      Eq. 17 is normalised by the same constant; with alpha in its numerator
      the normalised curve is F~ = d~^((3+k)/2).
  C2  Eq. 26 prints alpha Gamma Gamma in the numerator; F_crit = S d_crit with
      the flat-punch stiffness S of ``flat_punch_stiffness`` and d_crit of
      Eq. 25 (as printed) puts it in the denominator; at k = 0 this is
      Kendall's F = sqrt(8 pi gamma E* a^3).

The pressure fields of the graded Hertz and flat-punch contacts are not
printed in the paper (it cites them); they are restated here from the
Riesz-potential identity for the kernel r^-(1+k) and checked against Eq. 16
(corrected) by integration in the tests.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

from .bem_oracle import alpha, compliance


def gamma_pair(k: float) -> float:
    """Gamma((1+k)/2) Gamma((1-k)/2) = pi / cos(pi k / 2)."""
    return math.gamma((1.0 + k) / 2.0) * math.gamma((1.0 - k) / 2.0)


# ---- graded Hertz (paraboloid h = r^2 / 2R): Eqs. 14-17 -------------------

def hertz_depth(a: float, k: float, R: float) -> float:
    """Indentation depth d(a) of Eq. 15."""
    return a * a / ((1.0 + k) * R)


def hertz_radius(d: float, k: float, R: float) -> float:
    """Contact radius from Eq. 15 inverted."""
    return math.sqrt(max(d, 0.0) * (1.0 + k) * R)


def hertz_force(a: float, k: float, nu: float, R: float, E0: float = 1.0, c0: float = 1.0) -> float:
    """Normal force F(a) of Eq. 16, alpha in the denominator (C1)."""
    return 4.0 * E0 * a ** (3.0 + k) / (alpha(k, nu) * gamma_pair(k) * (1.0 + k) ** 2
                                        * (3.0 + k) * (1.0 - nu * nu) * c0 ** k * R)


def hertz_normalised(d: float, F: float, k: float, nu: float, R: float,
                     E0: float = 1.0, c0: float = 1.0):
    """Dimensionless (d~, F~) of Eq. 17 with alpha in the numerator (C1)."""
    dn = d / R
    Fn = gamma_pair(k) * (1.0 + k) ** 2 * (3.0 + k) * alpha(k, nu) * (1.0 - nu * nu) * c0 ** k \
        / (4.0 * (1.0 + k) ** ((3.0 + k) / 2.0) * R ** (2.0 + k) * E0) * F
    return dn, Fn


def hertz_deflection(r, a: float, k: float, R: float):
    """Surface deflection u_z(r, a) of Eq. 14 (B = non-regularised incomplete beta)."""
    r = np.asarray(r, dtype=np.float64)
    out = np.empty_like(r)
    inside = r < a
    out[inside] = (1.0 / (k + 1.0) - r[inside] ** 2 / (2.0 * a * a)) * a * a / R
    ro = r[~inside]
    x = (a / ro) ** 2

    def B(xx, p, q):
        return special.betainc(p, q, xx) * special.beta(p, q)

    val = math.cos(k * math.pi / 2.0) / (math.pi * (k + 1.0)) * (
        B(x, (1.0 + k) / 2.0, (1.0 - k) / 2.0)
        - (ro / a) ** 2 * B(x, (3.0 + k) / 2.0, (1.0 - k) / 2.0))
    out[~inside] = val * a * a / R
    return out


def hertz_pressure(r, a: float, k: float, nu: float, R: float, E0: float = 1.0, c0: float = 1.0):
    """Graded Hertz pressure p(r) = 2 cos(pi k/2) (a^2 - r^2)^((1+k)/2) / ((1+k)^2 R pi^2 A).

    Integrates to Eq. 16 (corrected, C1); at k = 0 it is Hertz's
    2 E* sqrt(a^2 - r^2) / (pi R).
    """
    r = np.asarray(r, dtype=np.float64)
    A = compliance(k, nu, E0, c0)
    s = np.clip(a * a - r * r, 0.0, None)
    return 2.0 * math.cos(math.pi * k / 2.0) * s ** ((1.0 + k) / 2.0) \
        / ((1.0 + k) ** 2 * R * math.pi ** 2 * A)


# ---- flat cylindrical punch -------------------------------------------------

def flat_punch_stiffness(a: float, k: float, nu: float, E0: float = 1.0, c0: float = 1.0) -> float:
    """S = dF/dd = 2 a^(1+k) / (A (1+k) Gamma((1+k)/2) Gamma((1-k)/2)); k = 0: 2 a E*."""
    return 2.0 * a ** (1.0 + k) / (compliance(k, nu, E0, c0) * (1.0 + k) * gamma_pair(k))


def flat_punch_pressure(r, a: float, d: float, k: float, nu: float, E0: float = 1.0,
                        c0: float = 1.0):
    """p(r) = p0 (1 - r^2/a^2)^(-(1-k)/2), p0 = d cos(pi k/2) / (A pi^2 a^(1-k))."""
    r = np.asarray(r, dtype=np.float64)
    A = compliance(k, nu, E0, c0)
    p0 = d * math.cos(math.pi * k / 2.0) / (A * math.pi ** 2 * a ** (1.0 - k))
    s = np.clip(1.0 - (r / a) ** 2, 1e-300, None)
    return np.where(r < a, p0 * s ** (-(1.0 - k) / 2.0), 0.0)


def flat_punch_dcrit(a: float, k: float, nu: float, dgamma: float, E0: float = 1.0,
                     c0: float = 1.0) -> float:
    """Critical separation distance of Eq. 25 (as printed)."""
    return math.sqrt(alpha(k, nu) * gamma_pair(k) * 2.0 * math.pi * (1.0 - nu * nu)
                     * dgamma * a ** (1.0 - k) * c0 ** k / E0)


def flat_punch_fcrit(a: float, k: float, nu: float, dgamma: float, E0: float = 1.0,
                     c0: float = 1.0) -> float:
    """Critical force of Eq. 26 with alpha Gamma Gamma in the denominator (C2)."""
    return math.sqrt(8.0 * math.pi * dgamma * E0 /
                     ((1.0 - nu * nu) * (1.0 + k) ** 2 * c0 ** k * alpha(k, nu) * gamma_pair(k))) \
        * a ** ((3.0 + k) / 2.0)


# ---- adhesive paraboloid (JKR-type), superposition of Hertz and flat punch --

def jkr_depth(a: float, k: float, nu: float, R: float, dgamma: float, E0: float = 1.0,
              c0: float = 1.0) -> float:
    """d(a) = a^2/((1+k)R) - d_crit(a): Eq. 15 minus the Eq. 25 flat-punch opening."""
    return hertz_depth(a, k, R) - flat_punch_dcrit(a, k, nu, dgamma, E0, c0)


def jkr_force(a: float, k: float, nu: float, R: float, dgamma: float, E0: float = 1.0,
              c0: float = 1.0) -> float:
    """F(a) = F_Hertz(a) - S(a) d_crit(a) (Eq. 16 corrected minus Eq. 26 corrected)."""
    return hertz_force(a, k, nu, R, E0, c0) - flat_punch_fcrit(a, k, nu, dgamma, E0, c0)


# ---- special cases of the influence coefficient ----------------------------

def love_rect(a0: float, a1: float, b0: float, b1: float) -> float:
    """k = 0: integral of 1/sqrt(a^2+b^2) over a rectangle (Love 1929, cited in Sec. 2.1).

    Corner sum of Phi(a, b), the integral over [0, a] x [0, b]: for a, b > 0
    Phi = a asinh(b/a) + b asinh(a/b), extended oddly in each argument.
    """
    def phi(a, b):
        if a == 0.0 or b == 0.0:
            return 0.0
        x, y = abs(a), abs(b)
        return math.copysign(1.0, a) * math.copysign(1.0, b) * (
            x * math.asinh(y / x) + y * math.asinh(x / y))
    return phi(a1, b1) - phi(a0, b1) - phi(a1, b0) + phi(a0, b0)


def eq11(k: float, q: float, p: float, n: float, m: float) -> float:
    """Closed form of Eq. 11 (Gauss hypergeometric functions), as printed.

    Valid when the element does not straddle the observation row or column.
    """
    F = special.hyp2f1
    e = (1.0 - k) / 2.0
    c = (k + 2.0) / 2.0
    t = (-n * p * (m * m + p * p) ** e * F(0.5, 1.0, c, -p * p / (m * m))
         + m * p * (n * n + p * p) ** e * F(0.5, 1.0, c, -p * p / (n * n))
         + n * q * (m * m + q * q) ** e * F(0.5, 1.0, c, -q * q / (m * m))
         - m * q * (n * n + q * q) ** e * F(0.5, 1.0, c, -q * q / (n * n))
         + k * n * p * (m * m + p * p) ** e * F(1.0, 1.0 - k / 2.0, 1.5, -p * p / (m * m))
         - k * m * p * (n * n + p * p) ** e * F(1.0, 1.0 - k / 2.0, 1.5, -p * p / (n * n))
         - k * n * q * (m * m + q * q) ** e * F(1.0, 1.0 - k / 2.0, 1.5, -q * q / (m * m))
         + k * m * q * (n * n + q * q) ** e * F(1.0, 1.0 - k / 2.0, 1.5, -q * q / (n * n)))
    return t / (m * n * (k - k * k))


def c1_k0_exact() -> float:
    """c1(0) = 4 ln(1 + sqrt 2) - 4 (sqrt 2 - 1) / 3 (mean of 1/r over two unit squares)."""
    return 4.0 * math.log(1.0 + math.sqrt(2.0)) - 4.0 * (math.sqrt(2.0) - 1.0) / 3.0
