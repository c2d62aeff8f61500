"""Physical pins of the oracle: hydrodynamic limits the paper derives, checked
on small periodic grids (no GPU).

* Sec. 4.1 / 4.4, Eq. (soundSpeed): the speed of sound is sqrt(gamma R T) of
  the mixture (not the isothermal sqrt(R T)); binary and ternary compositions,
  including S1 of Eq. (soundTestConditions).
* Sec. 3.3, Eq. (mu): a shear wave decays at nu k^2, nu = (1/omega - 1/2) R T,
  also in a frame moving along the wave vector (Galilean invariance, which the
  D3Q27 correction of Eq. fwithcorrection maintains).
* Sec. 2.3, Eqs. (constit2), (smDiffusionCoefficients2): a small binary
  mole-fraction wave decays at D_12 k^2, on the periodic grid and between
  the walls of the closed tube (Sec. 4.2), whose slowest mode places the
  walls halfway between the end nodes and their mirror images.
"""

import numpy as np
import pytest

import oracle as O


def _params(mm, cv, X0, T, mufac=0.1, D12=0.05, **kw):
    M = len(mm)
    mm = np.asarray(mm, float)
    cv = np.asarray(cv, float)
    D = np.full((M, M), D12)
    np.fill_diagonal(D, 0.0)
    mbar = float(np.dot(X0, mm))
    P0 = T / mbar
    mu = np.full(M, mufac * P0)
    lam = mu * (cv + 1.0) / mm / 0.71
    Y = np.asarray(X0) * mm / mbar
    return O.Params(mm, cv, D, mu=mu, lam=lam, slaved=int(np.argmax(Y)), **kw), P0


def _mixture_sound_speed(mm, cv, X0, T):
    mm, cv, X0 = (np.asarray(v, float) for v in (mm, cv, X0))
    mbar = float(np.dot(X0, mm))
    Y = X0 * mm / mbar
    cvm = float(np.dot(Y, cv / mm))
    R = 1.0 / mbar
    gamma = (cvm + R) / cvm
    return np.sqrt(gamma * R * T), np.sqrt(R * T)


@pytest.mark.parametrize("case", [
    ("He/Ar", [4.0, 40.0], [1.5, 1.5], [0.5, 0.5], 0.5, 0.02),
    ("S1 H2/Ar/CH4", [2.016, 39.948, 16.043], [2.5, 1.5, 3.0], [0.491, 0.509, 0.0], 0.5, 0.1),
    ("S2 H2/Ar/CH4", [2.016, 39.948, 16.043], [2.5, 1.5, 3.0], [0.2, 0.7, 0.1], 0.3, 0.1),
    ("H2/N2 cold", [2.0, 28.0], [2.5, 2.5], [0.3, 0.7], 0.2, 0.1),
])
def test_speed_of_sound(case):
    name, mm, cv, X0, T, mufac = case
    prm, P0 = _params(mm, cv, X0, T, mufac=mufac)
    n, steps = 64, 600
    M = len(mm)
    shape = (1, 1, n)
    x = np.arange(n)
    X = np.asarray(X0).reshape(M, 1, 1, 1) * np.ones((M,) + shape)
    P = P0 * (1.0 + 1e-4 * np.cos(2 * np.pi * x / n))[None, None, :]
    pops = O.init_populations(X, np.zeros((3,) + shape), np.full(shape, T), P, prm)
    amp = []
    for _ in range(steps):
        mom = O.moments(pops, prm)
        amp.append(np.dot(mom["j"][0, 0, 0] / mom["rho"][0, 0], np.sin(2 * np.pi * x / n)))
        pops = O.step(pops, prm)
    amp = np.array(amp)
    zc = [t + amp[t] / (amp[t] - amp[t + 1]) for t in range(5, steps - 1) if amp[t] * amp[t + 1] < 0]
    c_meas = n / (2.0 * np.mean(np.diff(zc)))
    cs, c_iso = _mixture_sound_speed(mm, cv, X0, T)
    assert abs(c_meas / cs - 1.0) < 5e-3, (name, c_meas, cs)
    assert abs(c_meas / c_iso - 1.0) > 0.05      # clearly not the isothermal speed


@pytest.mark.parametrize("ux0", [0.0, 0.05])
def test_shear_wave_viscosity(ux0):
    mm, cv, X0, T = [4.0, 40.0], [1.5, 1.5], [0.5, 0.5], 0.5
    prm, P0 = _params(mm, cv, X0, T, mufac=0.1)
    n, steps = 32, 300
    k = 2 * np.pi / n
    shape = (1, 1, n)
    x = np.arange(n)
    X = np.asarray(X0).reshape(2, 1, 1, 1) * np.ones((2,) + shape)
    u = np.zeros((3,) + shape)
    u[1] = 1e-3 * np.sin(k * x)
    u[0] = ux0
    pops = O.init_populations(X, u, np.full(shape, T), np.full(shape, P0), prm)
    mac = O.macroscopic(pops, prm)
    nu = float(((1.0 / mac["omega"] - 0.5) * mac["P"] / mac["rho"]).mean())     # Eq. (mu)
    amp = []
    for _ in range(steps):
        mom = O.moments(pops, prm)
        amp.append(np.abs(np.fft.rfft(mom["j"][1, 0, 0] / mom["rho"][0, 0])[1]))
        pops = O.step(pops, prm)
    rate = -np.log(amp[-1] / amp[50]) / (steps - 1 - 50)
    assert abs(rate / (nu * k * k) - 1.0) < 1.5e-2


@pytest.mark.parametrize("mm,cv,X1,D12", [([4.0, 40.0], [1.5, 1.5], 0.5, 0.05),
                                          ([2.0, 28.0], [2.5, 2.5], 0.3, 0.02)])
def test_binary_diffusion_rate(mm, cv, X1, D12):
    T = 0.5
    prm, P0 = _params(mm, cv, [X1, 1 - X1], T, mufac=0.1, D12=D12)
    n, steps = 32, 400
    k = 2 * np.pi / n
    shape = (1, 1, n)
    x = np.arange(n)
    X = np.empty((2,) + shape)
    X[0] = X1 + 1e-3 * np.cos(k * x)
    X[1] = 1 - X[0]
    pops = O.init_populations(X, np.zeros((3,) + shape), np.full(shape, T), np.full(shape, P0), prm)
    amp = []
    for _ in range(steps):
        mac = O.macroscopic(pops, prm)
        amp.append(np.abs(np.fft.rfft(mac["X"][0, 0, 0])[1]))
        pops = O.step(pops, prm)
    rate = -np.log(amp[-1] / amp[100]) / (steps - 1 - 100)
    assert abs(rate / (D12 * k * k) - 1.0) < 1.5e-2


def test_closed_tube_diffusion_rate():
    """Sec. 4.2 closed tube: between two walls the slowest composition mode is
    cos(k (x + 1/2)) with k = pi / n (no flux through walls halfway between
    the end nodes and their mirror images), and it decays at D_12 k^2 as the
    periodic mode does.  A wall placed on a node, or one that leaks, changes
    the rate."""
    T, D12, X1 = 0.5, 0.05, 0.5
    mm, cv = [4.0, 40.0], [1.5, 1.5]
    prm, P0 = _params(mm, cv, [X1, 1 - X1], T, mufac=0.1, D12=D12)
    prm.walls_x = True
    n, steps = 24, 400
    k = np.pi / n
    shape = (1, 1, n)
    x = np.arange(n)
    mode = np.cos(k * (x + 0.5))
    X = np.empty((2,) + shape)
    X[0] = X1 + 1e-3 * mode
    X[1] = 1 - X[0]
    pops = O.init_populations(X, np.zeros((3,) + shape), np.full(shape, T), np.full(shape, P0), prm)
    amp = []
    for _ in range(steps):
        mac = O.macroscopic(pops, prm)
        amp.append(float(np.dot(mac["X"][0, 0, 0] - X1, mode)))
        pops = O.step(pops, prm)
    rate = -np.log(amp[-1] / amp[100]) / (steps - 1 - 100)
    assert abs(rate / (D12 * k * k) - 1.0) < 1e-2, rate / (D12 * k * k)     # measured 1.0026
