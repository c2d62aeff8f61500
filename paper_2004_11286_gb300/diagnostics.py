"""Flow diagnostics of a state (host side, NumPy): the turbulent kinetic
energy spectrum of a periodic box and the slope of its inertial range, as
Sec. 4.5 uses to check the Kolmogorov -5/3 scaling of the Kelvin-Helmholtz
flow.  These read the observables (lbm_mix_get_moments); they are not part
of the step."""

from __future__ import annotations

import numpy as np


def tke_spectrum(u, rho=None, homogeneous=(0, 2)):
    """Shell-summed kinetic energy spectrum of the velocity fluctuations.

    u: (3, nz, ny, nx) velocity on a periodic box; rho: (nz, ny, nx) density
    (energy 1/2 rho |u'|^2, the density-weighted form of a compressible flow,
    with sqrt(rho) u' transformed) or None (1/2 |u'|^2).  The fluctuation is
    u minus its mean over the homogeneous axes (default z and x, the span and
    the stream of the shear layer; None: over the whole box).  Wavenumbers in units of 2 pi over the
    longest box edge; shells one unit of the shortest edge's fundamental
    wide.  Returns (k, E) with sum(E) the box mean of the fluctuating kinetic
    energy (Parseval)."""
    u = np.asarray(u, dtype=np.float64)
    _, nz, ny, nx = u.shape
    axes = tuple(range(1, 4)) if homogeneous is None else tuple(1 + a for a in homogeneous)
    up = u - u.mean(axis=axes, keepdims=True)
    w = up if rho is None else up * np.sqrt(np.asarray(rho, dtype=np.float64))[None]
    N = nz * ny * nx
    spec = 0.5 * sum(np.abs(np.fft.fftn(w[c])) ** 2 for c in range(3)) / N ** 2
    L = max(nz, ny, nx)
    kz = np.fft.fftfreq(nz) * nz * (L / nz)
    ky = np.fft.fftfreq(ny) * ny * (L / ny)
    kx = np.fft.fftfreq(nx) * nx * (L / nx)
    K = np.sqrt(kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2)
    width = L / min(nz, ny, nx)
    shell = np.rint(K / width).astype(np.int64)
    E = np.bincount(shell.ravel(), weights=spec.ravel())
    k = np.arange(E.size) * width
    return k, E


def spectral_slope(k, E, kmin, kmax):
    """Least-squares slope of log E against log k over kmin <= k <= kmax."""
    k, E = np.asarray(k), np.asarray(E)
    sel = (k >= kmin) & (k <= kmax) & (E > 0)
    if sel.sum() < 3:
        raise ValueError("fewer than three shells in the fit range")
    return float(np.polyfit(np.log(k[sel]), np.log(E[sel]), 1)[0])
