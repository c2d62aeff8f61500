"""Temperature-dependent specific heats (Sec. 3.1, Eqs. temperature, specUa,
specHa) on the GPU against the FP64 oracle with the same polynomials: the
per-node Newton solve of the temperature, the enthalpies H_a(T) in g^eq,
q^diff and q^corr (the last as sum_k T^k grad Phi_k of the mixture's
enthalpy coefficients), on random off-equilibrium states over both AA
parities; initialisation; and a constant polynomial against the
constant-heat path."""

import numpy as np
import pytest

import oracle as O
from paper_2004_11286_gb300 import workloads as W

from gpu_helpers import TOL, field_errors, gpu_handle, oracle_params, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2004_11286_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()


def _cs(wl):
    mbar = float(np.dot(wl.X.reshape(wl.M, -1).mean(axis=1), wl.molar_mass))
    return np.sqrt(1.4 * wl.T.mean() / mbar)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("M,coupling", [(2, "strong"), (3, "strong"), (3, "weak"), (8, "strong")])
def test_variable_heats_random_state_steps(M, coupling, precision):
    wl = W.random_mixture(M=M, shape=(5, 7, 12), seed=500 + M, velocity=0.03)
    cvp = W.variable_heats(wl.molar_mass, seed=M)
    prm = oracle_params(wl, coupling=coupling, cv_poly=cvp)
    pops = O.init_populations(wl.X, wl.u, wl.T, wl.P, prm) * W.perturbation((M + 2, 27) + wl.shape, 0.01, M)
    h = gpu_handle(wl, precision, coupling=coupling, cv_poly=cvp)
    h.set_populations(pops)
    ref = pops
    for k in range(3):
        ref = O.step(ref, prm)
        h.step(1)
        assert rel(h.populations(), ref) < TOL[precision], k
        mac = O.macroscopic(ref, prm)
        om = dict(rho=mac["rho"], u=mac["u"], T=mac["T"], P=mac["P"], X=mac["X"])
        errs = field_errors(h.moments_dict(), om, _cs(wl))
        assert max(errs.values()) < TOL[precision], (k, errs)
    h.close()


def test_variable_heats_init_fields_match_oracle():
    wl = W.random_mixture(M=3, shape=(3, 6, 11), seed=17, velocity=0.05)
    cvp = W.variable_heats(wl.molar_mass, seed=3)
    prm = oracle_params(wl, cv_poly=cvp)
    h = gpu_handle(wl, "fp64", cv_poly=cvp)
    h.init_fields(wl.X, wl.u, wl.T, wl.P)
    assert rel(h.populations(), O.init_populations(wl.X, wl.u, wl.T, wl.P, prm)) < 1e-14
    np.testing.assert_allclose(h.moments_dict()["T"], wl.T, rtol=1e-13)
    h.close()


def test_constant_polynomial_matches_constant_heats():
    wl = W.random_mixture(M=3, shape=(4, 5, 8), seed=19, velocity=0.02)
    a = gpu_handle(wl, "fp64")
    b = gpu_handle(wl, "fp64", cv_poly=wl.cv_molar[:, None])
    for h in (a, b):
        h.init_fields(wl.X, wl.u, wl.T, wl.P)
        h.step(10)
    assert rel(b.populations(), a.populations()) < 1e-13
    a.close()
    b.close()


def test_variable_heats_over_a_hundred_steps_fp32():
    """A smooth ternary mixture at rest with strongly T-dependent heats, 100
    steps: every field within the FP32 contract of the oracle."""
    wl = W.random_mixture(M=3, shape=(12, 12, 12), seed=21, amplitude=0.3)
    cvp = W.variable_heats(wl.molar_mass, seed=5)
    prm = oracle_params(wl, cv_poly=cvp)
    ref = O.run(O.init_populations(wl.X, wl.u, wl.T, wl.P, prm), prm, 100)
    h = gpu_handle(wl, "fp32", cv_poly=cvp)
    h.init_fields(wl.X, wl.u, wl.T, wl.P)
    h.step(100)
    mac = O.macroscopic(ref, prm)
    om = dict(rho=mac["rho"], u=mac["u"], T=mac["T"], P=mac["P"], X=mac["X"])
    errs = field_errors(h.moments_dict(), om, _cs(wl))
    assert max(errs.values()) < TOL["fp32"], errs
    h.close()
