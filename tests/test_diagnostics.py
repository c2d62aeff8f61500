"""The kinetic-energy spectrum diagnostic (paper_2004_11286_gb300.diagnostics)
against fields whose spectrum is known (no GPU): Parseval, a single Fourier
mode landing in its shell, and the slope of a synthetic field built with
E(k) ~ k^(-5/3)."""

import numpy as np

from paper_2004_11286_gb300.diagnostics import spectral_slope, tke_spectrum


def test_parseval_and_a_single_mode():
    nz, ny, nx = 8, 16, 16
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    u = np.zeros((3, nz, ny, nx))
    u[1] = 0.01 * np.cos(2 * np.pi * 3 * x / nx)          # |k| = 3 fundamentals of the longest edge
    k, E = tke_spectrum(u, homogeneous=None)
    assert np.isclose(E.sum(), 0.5 * (u ** 2).sum(axis=0).mean(), rtol=1e-12)
    i = int(np.argmax(E))
    assert abs(k[i] - 3.0) <= (k[1] - k[0]) / 2 and E[i] > 0.999 * E.sum()


def test_slope_of_a_kolmogorov_field():
    n = 64
    rng = np.random.Generator(np.random.PCG64(5))
    kf = np.fft.fftfreq(n) * n
    K = np.sqrt(kf[:, None, None] ** 2 + kf[None, :, None] ** 2 + kf[None, None, :] ** 2)
    amp = np.where(K > 0, K ** (-11.0 / 6.0), 0.0)       # |u_k|^2 ~ k^-11/3 -> E(k) ~ k^2 k^-11/3 = k^-5/3
    u = np.stack([np.real(np.fft.ifftn(amp * np.exp(2j * np.pi * rng.random((n, n, n))))) for _ in range(3)])
    k, E = tke_spectrum(u, homogeneous=None)
    assert abs(spectral_slope(k, E, 4, 24) + 5.0 / 3.0) < 0.1
