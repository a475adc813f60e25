"""Seeded synthetic inputs (no GPU)."""
import numpy as np
import pytest

from paper_1612_08395_gb300 import inputs as I


def test_paraboloid_centred_and_symmetric():
    h = I.paraboloid(8, R=2.0)
    assert h.min() == h[3, 3] == h[4, 4]
    np.testing.assert_array_equal(h, h[::-1, ::-1])
    np.testing.assert_array_equal(h, h.T)
    x = I.centres(8, 1 / 8)
    assert h[0, 0] == (x[0] ** 2 + x[0] ** 2) / 4.0


def test_flat_punch_area():
    h = I.flat_punch(256, 0.2)
    area = (h == 0).sum() / 256 ** 2
    assert abs(area - np.pi * 0.04) < 2 * np.pi * 0.2 / 256


def test_rough_surface_statistics_and_seed():
    h, zrms = I.rough_self_affine(256, hurst=0.8, q1_over_q0=32, rms_slope=0.1, seed=1612)
    h2, _ = I.rough_self_affine(256, hurst=0.8, q1_over_q0=32, rms_slope=0.1, seed=1612)
    np.testing.assert_array_equal(h, h2)
    assert h.min() == 0.0
    z = h.mean() - h  # h = max z - z and z has zero mean
    assert np.sqrt(np.mean(z ** 2)) == pytest.approx(zrms, rel=1e-12)
    gy, gx = np.gradient(z, 1 / 256)
    # spectral rms slope is 0.1; the finite-difference estimate is slightly lower
    assert 0.08 < np.sqrt(np.mean(gx ** 2 + gy ** 2)) < 0.1001
    # spectrum confined to the band q0..q1
    Z = np.abs(np.fft.rfft2(z))
    m = np.fft.fftfreq(256, 1 / 256)
    mr = np.fft.rfftfreq(256, 1 / 256)
    q = np.sqrt(mr[None, :] ** 2 + m[:, None] ** 2)
    assert Z[q > 32.5].max() < 1e-9 * Z.max()


def test_random_pressure_seeded():
    a = I.random_pressure(5, 7, seed=9, density=0.5)
    b = I.random_pressure(5, 7, seed=9, density=0.5)
    assert a.shape == (7, 5)
    np.testing.assert_array_equal(a, b)
    assert (a >= 0).all()
