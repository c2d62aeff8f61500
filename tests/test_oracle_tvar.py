"""Pins of the oracle's temperature-dependent specific heats (Sec. 3.1:
Eqs. eoscal, specUa, specHa, Umix, specH, temperature), no GPU.

The species' molar heat C-bar_{a,v}(T) / R_U is a polynomial in T (synthetic
coefficients of the form the NASA fits use; no thermochemical data exist
here).  Checked against what the mathematics fixes:
  * U_a(T) against numerical quadrature of C_{a,v}, H_a = U_a + R_a T;
  * the temperature solve of Eq. (temperature): the equilibrium state built
    from (X, u, T, P) returns its own T, to 1e-13;
  * a constant polynomial reproduces the constant-specific-heat method
    (Eq. temperature2) step for step, to rounding;
  * every collision still conserves species mass, momentum and energy;
  * the speed of sound is sqrt(gamma(T) R T) with gamma(T) = C_p(T)/C_v(T) at
    the local temperature (the adiabatic exponent of the ideal gas with
    temperature-dependent heats), not the constant-heat value;
  * isobaric, isothermal interdiffusion keeps T uniform (the enthalpies
    H_a(T) carried by the diffusion fluxes balance the internal energy, as
    in test_oracle_physics) with strongly T-dependent heats."""

import numpy as np
import pytest
from scipy.integrate import quad

import oracle as O

CV_POLY = np.array([[2.0, 2.5, 4.0],       # a diatomic-like heat rising with T
                    [1.5, 0.0, 0.0],       # monatomic, constant
                    [2.2, 5.0, -3.0]])     # polyatomic-like


def _params(M=3, **kw):
    mm = np.array([4.0, 40.0, 16.0])[:M]
    D = np.full((M, M), 0.05)
    np.fill_diagonal(D, 0.0)
    mu = np.full(M, 0.003)
    return O.Params(mm, CV_POLY[:M, 0], D, mu=mu, lam=mu * 5.0, cv_poly=CV_POLY[:M], slaved=1, **kw)


def test_internal_energy_and_enthalpy_are_the_integrals_of_the_heats():
    prm = _params()
    for T in (0.05, 0.2, 0.45):
        U = prm.U_a_of(np.array(T))
        H = prm.H_a_of(np.array(T))
        for a in range(3):
            q = quad(lambda t: float(prm.cv_a_of(np.array(t))[a]), 0.0, T, epsabs=1e-15, epsrel=1e-14)[0]
            assert np.isclose(U[a], q, rtol=1e-13)
            assert np.isclose(H[a], q + prm.R_a[a] * T, rtol=1e-13)


def test_temperature_solve_recovers_the_initial_temperature():
    prm = _params()
    rng = np.random.Generator(np.random.PCG64(4))
    shape = (3, 4, 5)
    X = rng.uniform(0.2, 1.0, (3,) + shape)
    X /= X.sum(axis=0)
    u = rng.uniform(-0.05, 0.05, (3,) + shape)
    T = rng.uniform(0.1, 0.4, shape)
    P = rng.uniform(0.01, 0.03, shape)
    st = O.node_state(O.moments(O.init_populations(X, u, T, P, prm), prm), prm)
    np.testing.assert_allclose(st["T"], T, rtol=1e-13)
    np.testing.assert_allclose(st["P"], P, rtol=1e-13)
    # C_p - C_v = R holds at every temperature (Mayer)
    np.testing.assert_allclose(st["Cp"] - st["Cv"], st["R"], rtol=1e-13)


def test_constant_polynomial_reproduces_the_constant_heat_method():
    base = _params()
    cv = np.array([2.5, 1.5, 3.0])
    p_const = O.Params(base.molar_mass, cv, base.D, mu=base.mu, lam=base.lam, slaved=1)
    p_poly = O.Params(base.molar_mass, cv, base.D, mu=base.mu, lam=base.lam, slaved=1, cv_poly=cv[:, None])
    rng = np.random.Generator(np.random.PCG64(8))
    shape = (4, 3, 5)
    X = rng.uniform(0.2, 1.0, (3,) + shape)
    X /= X.sum(axis=0)
    pops = O.init_populations(X, rng.uniform(-0.03, 0.03, (3,) + shape), np.full(shape, 0.3),
                              np.full(shape, 0.02), p_const)
    a, b = O.run(pops, p_const, 5), O.run(pops, p_poly, 5)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()


def test_collision_conserves_with_temperature_dependent_heats():
    prm = _params()
    rng = np.random.Generator(np.random.PCG64(9))
    shape = (3, 3, 4)
    X = rng.uniform(0.2, 1.0, (3,) + shape)
    X /= X.sum(axis=0)
    pops = O.init_populations(X, rng.uniform(-0.05, 0.05, (3,) + shape), rng.uniform(0.15, 0.35, shape),
                              rng.uniform(0.01, 0.03, shape), prm)
    pops = pops * (1.0 + 0.01 * rng.uniform(-1, 1, pops.shape))
    post = O.collide(pops, prm)
    d = (post - pops).sum(axis=1)                         # per node and lattice
    for a in range(3):
        if a != prm.slaved:
            assert np.abs(d[a]).max() < 1e-15 * 10
    assert np.abs(d[3]).max() < 1e-15 * 10               # mixture mass
    assert np.abs(d[4]).max() < 1e-14                    # total energy
    Cf = O.C.astype(float)
    dj = np.einsum("i...,id->d...", post[3] - pops[3], Cf).sum(axis=(1, 2, 3))
    assert np.abs(dj).max() < 1e-14                      # momentum (grid sum; the X term sums to zero)


def _sound_speed(prm, T0=0.4, n=64, steps=600):
    M = 2
    X0 = np.array([0.5, 0.5])
    P0 = T0 / float(np.dot(X0, prm.molar_mass))
    shape = (1, 1, n)
    x = np.arange(n)
    X = X0.reshape(M, 1, 1, 1) * np.ones((M,) + shape)
    P = P0 * (1.0 + 1e-4 * np.cos(2 * np.pi * x / n))[None, None, :]
    pops = O.init_populations(X, np.zeros((3,) + shape), np.full(shape, T0), P, prm)
    amp = []
    for _ in range(steps):
        mom = O.moments(pops, prm)
        amp.append(np.dot(mom["j"][0, 0, 0] / mom["rho"][0, 0], np.sin(2 * np.pi * x / n)))
        pops = O.step(pops, prm)
    amp = np.array(amp)
    zc = [t + amp[t] / (amp[t] - amp[t + 1]) for t in range(5, steps - 1) if amp[t] * amp[t + 1] < 0]
    return n / (2.0 * np.mean(np.diff(zc)))


def test_speed_of_sound_uses_the_local_adiabatic_exponent():
    """Sec. 4.1 / 4.4: a small sound wave sees the adiabatic exponent of the
    local temperature, gamma(T0) = C_p(T0) / C_v(T0), so the variable-heat
    mixture sounds like one with constant heats frozen at their T0 values
    (measured 0.02 % apart), and not like one with the heats at T = 0 (5 %
    faster).  Against sqrt(gamma(T0) R T0) the 64-cell wave is within 1 %
    (0.8 %, the lattice dispersion both constant-heat runs share)."""
    T0 = 0.4
    pv = _params(2)
    cv_T0 = pv.cv_a_of(np.array(T0)) * pv.molar_mass / pv.R_U
    frozen = O.Params(pv.molar_mass, cv_T0, pv.D, mu=pv.mu, lam=pv.lam, slaved=1)
    at_zero = O.Params(pv.molar_mass, CV_POLY[:2, 0], pv.D, mu=pv.mu, lam=pv.lam, slaved=1)
    c_var, c_frozen, c_zero = _sound_speed(pv, T0), _sound_speed(frozen, T0), _sound_speed(at_zero, T0)
    assert abs(c_var / c_frozen - 1.0) < 1e-3, (c_var, c_frozen)
    assert abs(c_zero / c_var - 1.0) > 0.03, (c_zero, c_var)
    mbar = float(np.dot([0.5, 0.5], pv.molar_mass))
    Y = 0.5 * pv.molar_mass / mbar
    cv = float(np.dot(Y, pv.cv_a_of(np.array(T0))))
    R = 1.0 / mbar
    assert abs(c_var / np.sqrt((cv + R) / cv * R * T0) - 1.0) < 1e-2


def test_interdiffusion_keeps_temperature_uniform_with_variable_heats():
    """As test_oracle_physics: He/Ar-like species (m = 4, 40), now with C-bar_v
    of the first rising with T; the enthalpy of each diffusing species is its
    own H_a(T).  Adiabatic part of the start-up sound wave removed with the
    local gamma(T0) (measured residual 1e-4; dropping q^diff gives 3e-2)."""
    mm, T0, n = np.array([4.0, 40.0]), 0.2, 32
    cvp = np.array([[1.5, 2.5, 4.0], [1.5, 0.0, 0.0]])
    X1, rho0 = 0.5, 2.0
    mbar = X1 * mm[0] + (1 - X1) * mm[1]
    P0 = rho0 * T0 / mbar
    mu = np.full(2, 0.1 * P0)
    prm = O.Params(mm, cvp[:, 0], np.array([[0.0, 0.05], [0.05, 0.0]]), mu=mu, lam=mu * 2.5 / mm / 0.71,
                   slaved=1, cv_poly=cvp)
    shape = (1, 1, n)
    X = np.empty((2,) + shape)
    X[0] = X1 + 0.05 * np.cos(2 * np.pi * np.arange(n) / n)
    X[1] = 1 - X[0]
    pops = O.init_populations(X, np.zeros((3,) + shape), np.full(shape, T0), np.full(shape, P0), prm)
    dev = 0.0
    for _ in range(300):
        pops = O.step(pops, prm)
        mac = O.macroscopic(pops, prm)
        Y = mac["Y"]
        cv = (Y * prm.cv_a_of(mac["T"])).sum(axis=0)
        R = 1.0 / (Y / mm.reshape(2, 1, 1, 1)).sum(axis=0) ** -1
        gam = (cv + R) / cv
        Ts = mac["T"] * (mac["P"] / P0) ** (-(gam - 1) / gam)
        dev = max(dev, float(np.abs(Ts / T0 - 1.0).max()))
    assert dev < 3e-4, dev
