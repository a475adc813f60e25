"""Seeded synthetic inputs: indenter profiles on the element grid.

This module holds no arithmetic of the contact method itself: it only lays out
indenter heights h(x, y) (the height of the indenter surface above its lowest
point, so h >= 0) on the element centres.  Both the CUDA path and the oracle
are fed from here.

Element centres: x_i = (i - N/2 + 1/2) dx, so the domain centre is a grid node
and centred indenters are symmetric under the grid's eight symmetries.

Profiles:
  paraboloid(N, R)            h = r^2 / (2R)                  (Sec. 2.2, Fig. 3)
  flat_punch(N, a)            h = 0 for r <= a, EXCLUDED else  (Sec. 3.2, Fig. 6)
  rough_self_affine(N, ...)   seeded self-affine random surface (Sec. 2.2, Fig. 4):
                              PSD ~ q^(-2(1+H)) between q0 and q1, random phases,
                              rms slope fixed; h = max z - z.

Request mixes (parameters only; profiles are built per job by job_profile):
  batch_jobs(count, seed)          independent solves of mixed size, k and adhesion
  serving_requests(count, seed)    the same kind of solves with Poisson arrival times

EXCLUDED (1e3, far above any indentation used) marks cells where the
indenter has no surface, so they can never come into contact.
"""
from __future__ import annotations

import numpy as np

EXCLUDED = 1.0e3


def centres(n: int, dx: float) -> np.ndarray:
    """Element centre coordinates (i - n/2 + 1/2) dx, i = 0..n-1."""
    return (np.arange(n) - n / 2.0 + 0.5) * dx


def radius_grid(nx: int, ny: int, dx: float, dy: float | None = None) -> np.ndarray:
    dy = dx if dy is None else dy
    x = centres(nx, dx)
    y = centres(ny, dy)
    return np.sqrt(x[None, :] ** 2 + y[:, None] ** 2)


def paraboloid(nx: int, R: float = 1.0, dx: float | None = None, ny: int | None = None) -> np.ndarray:
    """h = r^2/(2R) on an (ny, nx) grid, default domain side 1 (dx = 1/nx)."""
    ny = nx if ny is None else ny
    dx = 1.0 / nx if dx is None else dx
    r = radius_grid(nx, ny, dx)
    return r * r / (2.0 * R)


def flat_punch(nx: int, a: float, dx: float | None = None, ny: int | None = None) -> np.ndarray:
    """Flat cylindrical punch of radius a: h = 0 on r <= a, EXCLUDED outside."""
    ny = nx if ny is None else ny
    dx = 1.0 / nx if dx is None else dx
    r = radius_grid(nx, ny, dx)
    return np.where(r <= a, 0.0, EXCLUDED)


def square_punch(n: int, side: float, angle_deg: float = 0.0, dx: float | None = None) -> np.ndarray:
    """Flat square punch of the given side, rotated by angle_deg about the centre."""
    dx = 1.0 / n if dx is None else dx
    x = centres(n, dx)
    X, Y = np.meshgrid(x, x)
    c, s = np.cos(np.radians(angle_deg)), np.sin(np.radians(angle_deg))
    u = c * X + s * Y
    v = -s * X + c * Y
    inside = (np.abs(u) <= side / 2) & (np.abs(v) <= side / 2)
    return np.where(inside, 0.0, EXCLUDED)


def rough_self_affine(n: int, hurst: float = 0.8, q1_over_q0: float = 256.0,
                      rms_slope: float = 0.1, seed: int = 1612, L: float = 1.0):
    """Seeded self-affine surface; returns (h, rms_height_of_z).

    Modes q = 2 pi (mx, my) / L with q0 = 2 pi / L <= |q| <= q1 = q1_over_q0 q0
    get amplitude |q|^-(1+H) (so the PSD goes as q^-2(1+H)) and phases uniform in
    [0, 2 pi) from numpy's PCG64 with the given seed; the field is the real
    inverse transform (Hermitian by construction), has zero mean, and is scaled
    so that its rms gradient equals rms_slope.  h = max z - z >= 0.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    m = np.fft.fftfreq(n, d=1.0 / n)            # integer mode numbers
    mr = np.fft.rfftfreq(n, d=1.0 / n)
    MX, MY = np.meshgrid(mr, m)                 # shape (n, n//2+1)
    q = 2.0 * np.pi / L * np.sqrt(MX ** 2 + MY ** 2)
    q0 = 2.0 * np.pi / L
    q1 = q1_over_q0 * q0
    band = (q >= q0) & (q <= q1)
    amp = np.zeros_like(q)
    amp[band] = q[band] ** (-(1.0 + hurst))
    phase = rng.uniform(0.0, 2.0 * np.pi, size=q.shape)
    spec = amp * np.exp(1j * phase)
    spec[0, 0] = 0.0
    z = np.fft.irfft2(spec, s=(n, n))
    qx = 2.0 * np.pi / L * MX
    qy = 2.0 * np.pi / L * MY
    zx = np.fft.irfft2(1j * qx * spec, s=(n, n))
    zy = np.fft.irfft2(1j * qy * spec, s=(n, n))
    slope = np.sqrt(np.mean(zx ** 2 + zy ** 2))
    z *= rms_slope / slope
    z -= z.mean()
    h = z.max() - z
    return h, float(np.sqrt(np.mean(z ** 2)))


def random_pressure(nx: int, ny: int | None = None, seed: int = 0, density: float = 1.0) -> np.ndarray:
    """Seeded nonnegative random field for transform tests (uniform [0,1), a fraction zeroed)."""
    ny = nx if ny is None else ny
    rng = np.random.Generator(np.random.PCG64(seed))
    p = rng.random((ny, nx))
    if density < 1.0:
        p = np.where(rng.random((ny, nx)) < density, p, 0.0)
    return p


def _job(rng, n: int, index: int, seed_base: int) -> dict:
    """One solve: grid n x n on the unit square, k ~ U[-0.8, 0.8], nu = 0.3;
    paraboloid R = 1 (depth 0.01) or a rough surface (seed seed_base + index,
    q1 = 2 pi n / 16, depth = rms height); adhesive with probability 1/2, with
    dgamma log-uniform in [1e-4, 1e-2], preloaded to the depth and unloaded to
    d = 0 in 8 equal steps.  A non-adhesive job is one solve at the depth."""
    k = float(rng.uniform(-0.8, 0.8))
    rough = bool(rng.random() < 0.5)
    adhesive = bool(rng.random() < 0.5)
    dgamma = float(np.exp(rng.uniform(np.log(1e-4), np.log(1e-2)))) if adhesive else 0.0
    return {"n": int(n), "k": k, "nu": 0.3, "dgamma": dgamma, "adhesive": adhesive,
            "profile": "rough" if rough else "paraboloid", "seed": seed_base + index}


def job_profile(job: dict):
    """(h, d_steps) of a job from batch_jobs / serving_requests."""
    n = job["n"]
    if job["profile"] == "rough":
        h, depth = rough_self_affine(n, hurst=0.8, q1_over_q0=n / 16.0, rms_slope=0.1, seed=job["seed"])
    else:
        h, depth = paraboloid(n, 1.0), 0.01
    if job["adhesive"]:
        d_steps = depth * (1.0 - np.arange(9) / 8.0)
    else:
        d_steps = np.array([depth])
    return np.ascontiguousarray(h), d_steps


def batch_jobs(count: int = 256, seed: int = 4, sides=(128, 256, 512, 1024)) -> list:
    """count independent solves, grid side uniform over `sides`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    jobs = []
    for i in range(count):
        n = int(sides[rng.integers(len(sides))])
        jobs.append(_job(rng, n, i, 1000))
    return jobs


def serving_requests(count: int = 200, seed: int = 5, rate: float = 200.0,
                     n_min: int = 64, n_max: int = 2048) -> list:
    """count requests with Poisson arrivals (mean rate per second): each a job
    dict with an "arrival" time in seconds; grid side round(exp(U[ln n_min,
    ln n_max]))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        n = int(round(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))))
        job = _job(rng, n, i, 5000)
        job["arrival"] = t
        out.append(job)
    return out
