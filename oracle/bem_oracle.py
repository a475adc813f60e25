"""FP64 CPU oracle for the graded-material BEM contact solver.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the CPU
baseline / reference leg of ``bench.py`` may import this module.  It shares no
code with the CUDA library: no kernels, headers, tables or constants.  Its C
part (oracle_quad.c) is built by oracle/build.py.

Paper: Li & Popov, "Boundary element method for normal non-adhesive and
adhesive contacts of power-law graded elastic materials" (arXiv 1612.08395).
Each function names the equation or passage it follows.  Readings of the
paper where it is silent, garbled or inconsistent:

  R1  Eqs. 6, 8 and 23 print [(x-x')+(y-y')]^((1+k)/2); the integrand is
      [(x-x')^2+(y-y')^2]^((1+k)/2) as in Eq. 9 (the point-load kernel of
      Eq. 2 is r^-(1+k)).  The y-limits of Eqs. 6/8 use the y element size.
  R2  Eq. 13 drops the factor (1-nu^2) that Eqs. 2, 5, 7 and 12 carry; the
      prefactor A = alpha (1-nu^2) c0^k / E0 of Eq. 12 is used.
  R3  The conjugate-gradient inverse solve is only cited (Sec. 2.1, Polonsky &
      Keer).  It is read as the displacement-controlled Polonsky-Keer
      constrained CG: no mean-gap shift, no load rescale, initial pressure
      1e-3 on {h < d}, stopping rule sum|p - p_prev| / sum p < tol.
  R4  Detachment (Sec. 3.1, Eq. 24): "p > p_crit" means tensile stress, i.e.
      -p > p_crit with compressive p positive.  All violators detach at once,
      then the fixed-set problem is solved again; detached elements never
      re-attach while unloading.
  R5  c1(k) for k off the Table 1 grid: natural cubic spline of ln c1 through
      the 19 tabulated points.
  R6  Square elements are required for Eq. 24 (Sec. 3.1); non-square
      elements are allowed for the non-adhesive path.

Units: lengths in units of the domain side L, pressures in units of E0.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

_lib = None


def _clib():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_K_table.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_double, dp]
        lib.oracle_K_table.restype = ctypes.c_int
        lib.oracle_K_rect.argtypes = [ctypes.c_double] * 6 + [dp]
        lib.oracle_K_rect.restype = ctypes.c_double
        lib.oracle_c1_quad.argtypes = [ctypes.c_double, ctypes.c_double, dp]
        lib.oracle_c1_quad.restype = ctypes.c_double
        lib.oracle_direct_conv.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp, dp]
        lib.oracle_direct_conv.restype = None
        lib.oracle_direct_conv_at.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp,
                                              ctypes.c_int, ctypes.POINTER(ctypes.c_long), dp]
        lib.oracle_direct_conv_at.restype = None
        _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# --------------------------------------------------------------------------
# Material constants: Eqs. 2-4
# --------------------------------------------------------------------------

def beta(k: float, nu: float) -> float:
    """beta(k, nu) of Eq. 4."""
    return math.sqrt((1.0 + k) * (1.0 - k * nu / (1.0 - nu)))


def alpha(k: float, nu: float) -> float:
    """alpha(k, nu) of Eq. 3 (Gamma-function form as printed)."""
    b = beta(k, nu)
    num = (2.0 ** k) * b * math.sin(b * math.pi / 2.0) \
        * math.gamma((3.0 + k + b) / 2.0) * math.gamma((3.0 + k - b) / 2.0)
    den = math.sqrt(math.pi) * (1.0 + k) * math.cos(k * math.pi / 2.0) \
        * math.gamma(2.0 + k) * math.gamma(1.0 + k / 2.0) * math.gamma((1.0 - k) / 2.0)
    return num / den


def compliance(k: float, nu: float, E0: float = 1.0, c0: float = 1.0) -> float:
    """Prefactor A = alpha (1 - nu^2) c0^k / E0 of Eqs. 2, 7 and 12 (reading R2)."""
    return alpha(k, nu) * (1.0 - nu * nu) * c0 ** k / E0


# --------------------------------------------------------------------------
# Influence coefficients: Eqs. 7-10 (integrand of Eq. 9, reading R1)
# --------------------------------------------------------------------------

def influence_rect(k: float, a0: float, a1: float, b0: float, b1: float,
                   rel_tol: float = 1e-14) -> float:
    """Integral of (a^2+b^2)^(-(1+k)/2) over [a0,a1] x [b0,b1] (Eq. 9)."""
    return _clib().oracle_K_rect(k, a0, a1, b0, b1, rel_tol, None)


def influence_quarter(k: float, dx: float, dy: float, nx: int, ny: int,
                      rel_tol: float = 1e-14) -> np.ndarray:
    """K(di, dj) for 0 <= di < nx, 0 <= dj < ny as an (ny, nx) array (Eqs. 9-10).

    K depends only on the offsets (Eq. 10) and is even in each, so this
    quarter defines K for every offset pair.  Entry [dj, di] integrates over
    a in [(di-1/2)dx, (di+1/2)dx], b in [(dj-1/2)dy, (dj+1/2)dy].
    """
    out = np.empty((ny, nx), dtype=np.float64)
    rc = _clib().oracle_K_table(k, dx, dy, nx, ny, rel_tol, _dptr(out))
    if rc != 0:
        raise RuntimeError("oracle cubature failed")
    return out


def c1_uncorrected(k: float, rel_tol: float = 1e-13) -> float:
    """c1(k) of Eq. 23 (integrand per reading R1) by cubature."""
    return _clib().oracle_c1_quad(k, rel_tol, None)


# Table 1 (Sec. 3.1): corrected c1(k).  Typed from the paper.
TABLE1_K = np.array([-0.9, -0.8, -0.7, -0.6, -0.5, -0.4, -0.3, -0.2, -0.1, 0.0,
                     0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9])
TABLE1_C1 = np.array([0.14, 0.31, 0.495, 0.71, 0.96, 1.24, 1.58, 1.97, 2.43, 2.97,
                      3.66, 4.52, 5.62, 7.10, 9.15, 12.25, 17.50, 27.65, 58.00])


def _natural_spline_second_derivs(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Second derivatives of the natural cubic spline through (x, y)."""
    n = len(x)
    h = np.diff(x)
    a = np.zeros((n, n))
    rhs = np.zeros(n)
    a[0, 0] = a[-1, -1] = 1.0
    for i in range(1, n - 1):
        a[i, i - 1] = h[i - 1]
        a[i, i] = 2.0 * (h[i - 1] + h[i])
        a[i, i + 1] = h[i]
        rhs[i] = 6.0 * ((y[i + 1] - y[i]) / h[i] - (y[i] - y[i - 1]) / h[i - 1])
    return np.linalg.solve(a, rhs)


def c1_corrected(k: float) -> float:
    """Corrected c1(k): Table 1 on its grid, natural cubic spline of ln c1 between (R5)."""
    if not (-0.9 <= k <= 0.9):
        raise ValueError("corrected c1 is tabulated for -0.9 <= k <= 0.9 only")
    x, y = TABLE1_K, np.log(TABLE1_C1)
    m = _natural_spline_second_derivs(x, y)
    i = int(np.clip(np.searchsorted(x, k) - 1, 0, len(x) - 2))
    h = x[i + 1] - x[i]
    s = (k - x[i]) / h
    val = (1 - s) * y[i] + s * y[i + 1] \
        + h * h / 6.0 * (((1 - s) ** 3 - (1 - s)) * m[i] + (s ** 3 - s) * m[i + 1])
    return float(math.exp(val))


def p_crit(k: float, nu: float, dgamma: float, delta: float,
           E0: float = 1.0, c0: float = 1.0, c1: float | None = None) -> float:
    """Critical tensile stress of Eq. 24 for square elements of side delta."""
    if c1 is None:
        c1 = c1_corrected(k)
    return math.sqrt(2.0 * E0 * dgamma /
                     (alpha(k, nu) * (1.0 - nu * nu) * c1 * c0 ** k * delta ** (1.0 - k)))


# --------------------------------------------------------------------------
# The stress -> displacement transform: Eq. 7/12 (direct) and Eq. 13 (FFT)
# --------------------------------------------------------------------------

def convolve_direct(Kq: np.ndarray, p: np.ndarray) -> np.ndarray:
    """sum_{i'j'} K(i-i', j-j') p_{i'j'} by the direct O(N^4) sum (Eq. 7).

    Kq[dj, di] must cover 0 <= dj < ny, 0 <= di < nx for p of shape (ny, nx).
    """
    ny, nx = p.shape
    Kq = np.ascontiguousarray(Kq, dtype=np.float64)
    if Kq.shape[0] < ny or Kq.shape[1] < nx:
        raise ValueError("influence table too small")
    p = np.ascontiguousarray(p, dtype=np.float64)
    u = np.empty_like(p)
    _clib().oracle_direct_conv(nx, ny, _dptr(Kq), Kq.shape[1], _dptr(p), _dptr(u))
    return u


def convolve_direct_at(Kq: np.ndarray, p: np.ndarray, flat_idx: np.ndarray) -> np.ndarray:
    """The direct sum of Eq. 7 at selected flat output indices iy*nx + ix."""
    ny, nx = p.shape
    Kq = np.ascontiguousarray(Kq, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    idx = np.ascontiguousarray(flat_idx, dtype=np.int64)
    out = np.empty(len(idx), dtype=np.float64)
    _clib().oracle_direct_conv_at(nx, ny, _dptr(Kq), Kq.shape[1], _dptr(p), len(idx),
                                  idx.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _dptr(out))
    return out


def torus_kernel(Kq: np.ndarray, py: int, px: int) -> np.ndarray:
    """Even extension of the quarter table onto a py x px torus.

    Offset (y, x) on the torus is the signed offset (min(y, py-y), min(x, px-x));
    every torus offset holds its true K value (the quarter must reach py/2, px/2).
    """
    iy = np.minimum(np.arange(py), py - np.arange(py))
    ix = np.minimum(np.arange(px), px - np.arange(px))
    if Kq.shape[0] <= iy.max() or Kq.shape[1] <= ix.max():
        raise ValueError("influence table too small for the torus")
    return Kq[np.ix_(iy, ix)]


class FFTConvolver:
    """u = K * p by FFT on the zero-padded (2ny) x (2nx) torus (Eq. 13).

    A library FP64 FFT is the step: numpy's by default, scipy.fft's with
    `workers` threads when workers != 1 (the same real 2D transforms, run on
    several host cores).  The spectrum FFT(K) is taken once.  Kq must cover
    offsets 0..ny and 0..nx.
    """

    def __init__(self, Kq: np.ndarray, ny: int, nx: int, workers: int = 1):
        self.ny, self.nx = ny, nx
        self.py, self.px = 2 * ny, 2 * nx
        self.workers = workers
        self.khat = self._rfft2(torus_kernel(Kq, self.py, self.px))

    def _rfft2(self, x):
        if self.workers == 1:
            return np.fft.rfft2(x)
        import scipy.fft
        return scipy.fft.rfft2(x, workers=self.workers)

    def _irfft2(self, X):
        if self.workers == 1:
            return np.fft.irfft2(X, s=(self.py, self.px))
        import scipy.fft
        return scipy.fft.irfft2(X, s=(self.py, self.px), workers=self.workers)

    def __call__(self, p: np.ndarray) -> np.ndarray:
        pad = np.zeros((self.py, self.px))
        pad[:self.ny, :self.nx] = p
        u = self._irfft2(self._rfft2(pad) * self.khat)
        return u[:self.ny, :self.nx]


class DirectConvolver:
    """u = K * p by the direct sum of Eq. 7."""

    def __init__(self, Kq: np.ndarray, ny: int, nx: int):
        self.Kq = np.ascontiguousarray(Kq[:ny, :nx])

    def __call__(self, p: np.ndarray) -> np.ndarray:
        return convolve_direct(self.Kq, p)


# --------------------------------------------------------------------------
# Non-adhesive inverse problem (Sec. 2.1, reading R3)
# --------------------------------------------------------------------------

class SolveResult:
    def __init__(self, **kw):
        self.__dict__.update(kw)


def pk_solve(A: float, conv, h: np.ndarray, d: float, p0: np.ndarray | None = None,
             tol: float = 1e-10, max_iter: int = 10000) -> SolveResult:
    """Polonsky-Keer constrained CG for p >= 0, g >= 0, p g = 0 with g = A K p + h - d.

    Steps in order (reading R3 of the cited algorithm):
      1 g = A K*p + h - d          2 Ic = {p > 0}       3 G = sum_Ic g^2
      4 t = g + delta (G/G_old) t on Ic, else 0; G_old = G
      5 r = A K*t                   6 tau = sum_Ic g t / sum_Ic r t
      7 p <- max(p - tau t, 0) on Ic
      8 Iol = {p = 0, g < 0}: if empty delta = 1, else delta = 0 and p = -tau g on Iol
      9 eps = sum |p - p_prev| / sum p; stop when eps < tol
    """
    h = np.asarray(h, dtype=np.float64)
    if p0 is None:
        p = np.where(h < d, 1e-3, 0.0)
    else:
        p = np.array(p0, dtype=np.float64)
    delta, G_old = 0.0, 1.0
    t = np.zeros_like(p)
    eps = math.inf
    it = 0
    g = A * conv(p) + h - d
    while it < max_iter:
        Ic = p > 0
        if not Ic.any():
            # no element in contact: the indenter is separated (or all pressure
            # projected out); the overlap step below can re-activate elements
            if (g < 0).any():
                p = np.where(g < 0, 1e-3, 0.0)
                g = A * conv(p) + h - d
                it += 1
                continue
            eps = 0.0
            break
        G = float(np.sum(g[Ic] ** 2))
        t = np.where(Ic, g + delta * (G / G_old) * t, 0.0)
        G_old = G
        r = A * conv(t)
        rt = float(np.sum(r[Ic] * t[Ic]))
        if G == 0.0 or rt == 0.0:
            eps = 0.0
            break
        tau = float(np.sum(g[Ic] * t[Ic])) / rt
        p_prev = p
        p = np.where(Ic, p - tau * t, p)
        p = np.maximum(p, 0.0)
        Iol = (p == 0.0) & (g < 0.0)
        if Iol.any():
            delta = 0.0
            p = np.where(Iol, -tau * g, p)
        else:
            delta = 1.0
        it += 1
        sp = float(np.sum(p))
        eps = float(np.sum(np.abs(p - p_prev))) / sp if sp > 0 else 0.0
        g = A * conv(p) + h - d
        if eps < tol:
            break
    return SolveResult(p=p, g=g, iterations=it, eps=eps, converged=eps < tol)


# --------------------------------------------------------------------------
# Adhesive contact (Sec. 3.1, Eq. 24 and the algorithm that follows it)
# --------------------------------------------------------------------------

def fixed_set_cg(A: float, conv, c: np.ndarray, S: np.ndarray, p0: np.ndarray,
                 tol: float = 1e-12, max_iter: int = 100000) -> SolveResult:
    """Solve A (K p)_S + c_S = 0 with p = 0 off S by plain conjugate gradients.

    This is the fixed-contact-area step of the adhesive algorithm: the contact
    area is held, tension is allowed inside it.  c = h - d.  Stops when the
    residual norm falls below tol times the norm of c on S.
    """
    S = np.asarray(S, dtype=bool)
    p = np.where(S, p0, 0.0)
    if not S.any():
        return SolveResult(p=p, iterations=0, residual=0.0, converged=True)
    g = np.where(S, A * conv(p) + c, 0.0)
    bnorm = float(np.linalg.norm(c[S]))
    bnorm = bnorm if bnorm > 0 else 1.0
    t = g.copy()
    G = float(np.sum(g * g))
    it = 0
    while it < max_iter and math.sqrt(G) > tol * bnorm:
        r = np.where(S, A * conv(t), 0.0)
        tr = float(np.sum(t * r))
        if tr <= 0.0:
            break
        tau = G / tr
        p = p - tau * t
        g = g - tau * r
        G_new = float(np.sum(g * g))
        t = g + (G_new / G) * t
        G = G_new
        it += 1
    return SolveResult(p=p, iterations=it, residual=math.sqrt(G) / bnorm,
                       converged=math.sqrt(G) <= tol * bnorm)


def adhesive_unload(A: float, conv, h: np.ndarray, d0: float, d_steps, pcrit: float,
                    cell_area: float, tol_pk: float = 1e-10, tol_cg: float = 1e-12,
                    p_init: np.ndarray | None = None, S_init: np.ndarray | None = None):
    """Adhesive pull-off (Sec. 3.1, after Eq. 24; readings R4).

    Preload non-adhesively to d0 (unless a state p_init/S_init is given), then
    for each depth d in d_steps: hold the contact area, solve for p, detach
    every element with -p > pcrit at once, and repeat until none detaches.
    Returns per-step dicts (d, force, area, count, rounds) and the final p, S.
    """
    if p_init is None:
        pre = pk_solve(A, conv, h, d0, tol=tol_pk)
        p = pre.p
        S = p > 0
    else:
        p = np.array(p_init, dtype=np.float64)
        S = np.array(S_init, dtype=bool)
    out = []
    for d in d_steps:
        rounds = 0
        iters = 0
        while True:
            res = fixed_set_cg(A, conv, h - d, S, p, tol=tol_cg)
            p = res.p
            iters += res.iterations
            D = S & (-p > pcrit)
            if not D.any():
                break
            S = S & ~D
            p = np.where(S, p, 0.0)
            rounds += 1
        out.append(dict(d=float(d), force=cell_area * float(np.sum(p)),
                        area=cell_area * int(S.sum()), count=int(S.sum()),
                        rounds=rounds, iterations=iters))
    return out, p, S
