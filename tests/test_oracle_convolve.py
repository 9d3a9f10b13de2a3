"""Pins of the oracle's Gaussian convolution and statistical averaging."""
import math

import numpy as np

from oracle import rmatrix as o


def gauss(x, mu, sd):
    return np.exp(-0.5 * ((x - mu) / sd) ** 2) / (sd * math.sqrt(2 * math.pi))


def test_gaussian_widths_add_in_quadrature():
    E = np.linspace(0.0, 2.0, 4001)
    s1, fwhm = 0.03, 0.05
    s2 = fwhm / (2 * math.sqrt(2 * math.log(2)))
    out = o.convolve_average(E, gauss(E, 1.0, s1)[None, :], [1.0], fwhm)
    want = gauss(E, 1.0, math.hypot(s1, s2))
    inner = (E > 0.5) & (E < 1.5)
    assert np.abs(out[inner] - want[inner]).max() <= 1e-10 * want.max()


def test_constant_stays_constant_and_area_is_kept():
    rng = np.random.default_rng(3)
    E = np.sort(rng.uniform(0.0, 3.0, 3000))  # a non-uniform mesh
    assert np.allclose(o.convolve_average(E, np.full((1, E.size), 2.5), [1.0], 0.07), 2.5, rtol=1e-14)
    # on a uniform mesh the normalised kernel is symmetric, so the area of a peak away from the
    # ends is kept
    E = np.linspace(0.0, 3.0, 3001)
    sig = gauss(E, 1.5, 0.02)
    out = o.convolve_average(E, sig[None, :], [1.0], 0.04)
    tw = o.trapezoid_weights(E)
    assert abs(np.dot(tw, out) - np.dot(tw, sig)) <= 1e-12 * np.dot(tw, sig)


def test_narrow_kernel_returns_the_input():
    E = np.linspace(0.0, 1.0, 501)
    sig = np.sin(7 * E) ** 2
    out = o.convolve_average(E, sig[None, :], [1.0], 1e-6)  # far below the 2e-3 spacing
    assert np.abs(out - sig).max() <= 1e-12


def test_statistical_average_is_linear():
    E = np.linspace(0.0, 1.0, 301)
    a, b = np.cos(5 * E) ** 2, np.exp(-E)
    both = o.convolve_average(E, np.vstack([a, b]), [2 / 3, 1 / 3], 0.02)
    sep = (2 / 3) * o.convolve_average(E, a[None, :], [1.0], 0.02) + (1 / 3) * o.convolve_average(E, b[None, :], [1.0], 0.02)
    assert np.abs(both - sep).max() <= 1e-14
    assert np.allclose(o.convolve_average(E, np.vstack([a, b]), [0.25, 0.75], 0.0), 0.25 * a + 0.75 * b, rtol=1e-15)


def test_nonuniform_mesh_uses_trapezoid_weights():
    # points twice as dense on one side: the closed form holds only with the mesh weights
    u = np.linspace(0.0, 1.0, 6001)
    E = 2.0 * u ** 2  # spacing grows linearly
    s1, fwhm = 0.03, 0.05
    s2 = fwhm / (2 * math.sqrt(2 * math.log(2)))
    out = o.convolve_average(E, gauss(E, 1.0, s1)[None, :], [1.0], fwhm)
    want = gauss(E, 1.0, math.hypot(s1, s2))
    inner = (E > 0.6) & (E < 1.4)
    assert np.abs(out[inner] - want[inner]).max() <= 2e-5 * want.max()
