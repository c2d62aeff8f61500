"""Physics of the GPU step, independent of the oracle: the speed of sound of
the binary acoustic pulse at the benchmark's full size (128^3, m = 4, 40,
FP32, 2000 steps) for mole fractions 0.2, 0.5 and 0.8 against the mixture's
ideal-gas closed form sqrt(gamma R T) (Secs. 4.1, 4.4, Eq. soundSpeed); and
the osmotic-diffusion transient of the closed ternary tube against the
linearised Maxwell-Stefan theory (Sec. 4.2)."""

import numpy as np
import pytest

from paper_2004_11286_gb300 import workloads as W

from gpu_helpers import gpu_handle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2004_11286_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()


def _closed_form(wl):
    X0 = wl.X[:, 0, 0, 0]
    mbar = float(np.dot(X0, wl.molar_mass))
    Y = X0 * wl.molar_mass / mbar
    cv = float(np.dot(Y, wl.cv_molar / wl.molar_mass))     # R_U = 1
    R = 1.0 / mbar
    T = float(wl.T.mean())
    return np.sqrt((cv + R) / cv * R * T), np.sqrt(R * T)


def _mode_frequency(a, t, omega0):
    """Angular frequency of one standing Fourier mode a(t) = A cos(omega t +
    phi) exp(-gamma t) + B (B: the slow non-acoustic part)."""
    from scipy.optimize import curve_fit

    def model(t, A, om, g, ph, B):
        return A * np.cos(om * t + ph) * np.exp(-g * t) + B

    p0 = (float(np.abs(a).max()), omega0, 1e-4, 0.0, 0.0)
    (A, om, g, ph, B), _ = curve_fit(model, t, a, p0=p0, maxfev=50000)
    return abs(om)


@pytest.mark.parametrize("x1", [0.2, 0.5, 0.8])
def test_acoustic_pulse_speed_of_sound(x1):
    """The pressure averaged over y-z planes of the spherical pulse obeys the
    1-D wave equation, so each of its Fourier modes along x is a standing wave
    cos(omega(k) t).  The phase speed omega / k of the longest modes,
    extrapolated to k -> 0 (the lattice's dispersion is even in k), is the
    speed of sound; the pulse itself (width 6 cells, k sigma ~ 1) travels a
    little slower, by the same dispersion."""
    import torch
    wl = W.acoustic_pulse(x1=x1)
    nz, ny, nx = wl.shape
    cs, c_iso = _closed_form(wl)
    h = gpu_handle(wl, "fp32")
    h.init_fields(wl.X, wl.u, wl.T, wl.P)
    buf = torch.empty(h.n_outputs * h.N, dtype=torch.float64, device="cuda")
    every, steps = 10, 2000
    prof, times = [], []
    for t in range(0, steps + 1, every):
        if t:
            h.step(every)
        h.moments(out=buf)
        prof.append(buf.view(h.n_outputs, nz, ny, nx)[5].mean(dim=(0, 1)).cpu().numpy())
        times.append(float(t))
    h.close()
    prof = np.array(prof)
    times = np.array(times)
    # the pulse is centred on x = nx / 2: the modes' coefficients are real up to (-1)^m
    modes = np.fft.rfft(prof - prof.mean(axis=1, keepdims=True), axis=1)
    speeds = []
    for m in (1, 2, 3):
        k = 2.0 * np.pi * m / nx
        a = (modes[:, m] * np.exp(1j * k * (nx / 2))).real
        speeds.append(_mode_frequency(a, times, cs * k) / k)
    ks = 2.0 * np.pi * np.arange(1, 4) / nx
    c0, curv = np.polynomial.polynomial.polyfit(ks ** 2, speeds, 1)
    assert abs(c0 / cs - 1.0) < 5e-3, (x1, c0, cs, speeds)
    assert abs(speeds[0] / cs - 1.0) < 1e-2, (x1, speeds, cs)
    assert speeds[0] > speeds[1] > speeds[2]        # normal dispersion: shorter waves are slower
    assert abs(c0 / c_iso - 1.0) > 0.1              # the adiabatic, not the isothermal speed


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_closed_tube_osmotic_diffusion_transient(precision):
    """Sec. 4.2: the closed H2/Ar/CH4 tube (64 x 4 x 4, walls on both x
    faces), 40000 steps: hydrogen, at the same mole fraction in both halves,
    builds up a half-tube difference and loses it again (osmotic diffusion).
    Its whole transient, and the argon and methane differences, follow the
    linearised Maxwell-Stefan theory."""
    from ms_theory import half_tube_differences, osmotic_tube
    from paper_2004_11286_gb300 import binding
    L, steps, every = 64, 40000, 4000
    X0, D = osmotic_tube(L)
    mm, cv = np.array([2.0, 40.0, 16.0]), np.array([2.5, 1.5, 3.0])
    T = 0.2
    P0 = T / float(np.dot(X0.mean(axis=1), mm))
    mu = np.full(3, 0.1 * P0)
    shape = (4, 4, L)
    h = binding.LbmMix(mm, cv, D, mu=mu, lam=mu * (cv + 1.0) / mm / 0.71, shape=shape, precision=precision,
                       slaved=1, walls_x=True)
    X = np.broadcast_to(X0[:, None, None, :], (3,) + shape).copy()
    h.init_fields(X, np.zeros((3,) + shape), np.full(shape, T), np.full(shape, P0))
    times, sim = [], []
    for t in range(every, steps + 1, every):
        h.step(every)
        Xs = h.moments_dict()["X"].mean(axis=(1, 2))
        sim.append(Xs[:, :L // 2].mean(axis=1) - Xs[:, L // 2:].mean(axis=1))
        times.append(t)
    h.close()
    sim = np.array(sim)
    th = half_tube_differences(X0, D, times)
    peak = float(th[:, 0].max())
    k = int(np.argmax(sim[:, 0]))
    assert 0 < k < len(times) - 1                                    # rises, then falls
    assert np.abs(sim[:, 0] - th[:, 0]).max() < 0.03 * peak, (sim[:, 0], th[:, 0])
    d0 = X0[1, :L // 2].mean() - X0[1, L // 2:].mean()
    assert np.abs(sim[:, 1:] - th[:, 1:]).max() < 0.01 * d0, (sim[:, 1:], th[:, 1:])
