"""Bounce-back walls normal to x (the closed tube of Sec. 4.2) on the GPU
against the FP64 oracle's walls: every lattice reflected halfway, the
deferred non-local terms of reflected populations, the mirror rule of the
isotropic derivative at the walls (per-node and row-blocked stencils, the
runtime species loop of M >= 4), both AA parities, and the readers."""

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


def _moments(pops, prm):
    mac = O.macroscopic(pops, prm)
    return dict(rho=mac["rho"], u=mac["u"], T=mac["T"], P=mac["P"], X=mac["X"])


# (5, 7, 13): per-node stencils; (4, 5, 8): row-blocked stencils; (3, 2, 1): both walls at one node.
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(5, 7, 13), (4, 5, 8), (3, 2, 1)])
@pytest.mark.parametrize("M,coupling", [(3, "strong"), (2, "weak"), (8, "strong")])
def test_walled_random_state_steps(M, coupling, shape, precision):
    wl = W.random_mixture(M=M, shape=shape, seed=300 + M, velocity=0.03)
    prm = oracle_params(wl, coupling=coupling, walls_x=True)
    pops = O.init_populations(wl.X, wl.u, wl.T, wl.P, prm) * W.perturbation((M + 2, 27) + shape, 0.01, M)
    h = gpu_handle(wl, precision, coupling=coupling, walls_x=True)
    h.set_populations(pops)
    ref = pops
    for k in range(4):                       # parities 0, 1, 0, 1
        ref = O.step(ref, prm)
        h.step(1)
        assert rel(h.populations(), ref) < TOL[precision], k
        errs = field_errors(h.moments_dict(), _moments(ref, prm), _cs(wl))
        assert max(errs.values()) < TOL[precision], (k, errs)
    h.close()


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
@pytest.mark.parametrize("shape", [(5, 7, 13), (4, 5, 8)])
def test_walled_reduced_precision_steps(shape, precision):
    """16-bit storage with walls: a population reflected at a wall was stored
    against the node's own equilibrium for the opposite direction, and is
    decoded with it (both parities).  A smooth ternary state at rest with
    0.2 % population noise; every field within 1e-3, u with the floor of
    the other 16-bit tests (BF16 holds the interdiffusion drift to a few
    1e-3 of the 1e-3 c_s floor)."""
    wl = W.random_mixture(M=3, shape=shape, seed=303)
    prm = oracle_params(wl, walls_x=True)
    pops = O.init_populations(wl.X, wl.u, wl.T, wl.P, prm) * W.perturbation((5, 27) + shape, 0.002, 3)
    h = gpu_handle(wl, precision, walls_x=True)
    h.set_populations(pops)
    ref = pops
    for k in range(4):
        ref = O.step(ref, prm)
        h.step(1)
        errs = field_errors(h.moments_dict(), _moments(ref, prm), _cs(wl))
        assert max(v for f, v in errs.items() if f != "u") < 1e-3, (k, errs)
        assert errs["u"] < (1e-3 if precision == "fp16" else 6e-3), (k, errs)
    h.close()


def test_walls_change_the_result():
    # the same state on the periodic grid differs: the walls are in effect
    wl = W.random_mixture(M=3, shape=(4, 5, 8), seed=303, velocity=0.03)
    hw = gpu_handle(wl, "fp64", walls_x=True)
    hp = gpu_handle(wl, "fp64")
    for h in (hw, hp):
        h.init_fields(wl.X, wl.u, wl.T, wl.P)
        h.step(3)
    assert rel(hw.populations(), hp.populations()) > 1e-6
    hw.close()
    hp.close()


def test_walled_state_set_at_odd_parity_roundtrips():
    wl = W.random_mixture(M=3, shape=(4, 3, 6), seed=310, velocity=0.03)
    prm = oracle_params(wl, walls_x=True)
    h = gpu_handle(wl, "fp64", walls_x=True)
    h.init_fields(wl.X, wl.u, wl.T, wl.P)
    h.step(1)                                # the state is now stored at the odd parity
    ref = O.step(O.init_populations(wl.X, wl.u, wl.T, wl.P, prm), prm)
    ref = ref * W.perturbation(ref.shape, 0.01, 7)
    h.set_populations(ref)
    assert rel(h.populations(), ref) < 1e-15
    h.step(3)
    assert rel(h.populations(), O.run(ref, prm, 3)) < TOL["fp64"]
    h.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_closed_box_conserves_on_gpu(precision):
    wl = W.random_mixture(M=3, shape=(6, 5, 8), seed=320, velocity=0.03)
    prm = oracle_params(wl, walls_x=True)
    h = gpu_handle(wl, precision, walls_x=True)
    h.init_fields(wl.X, wl.u, wl.T, wl.P)
    s0 = h.diagnostics()
    h.step(41)
    s1 = h.diagnostics()
    keep = [a for a in range(3) if a != prm.slaved] + [3, 7]   # unslaved species, rho, rho E
    np.testing.assert_allclose(s1[keep], s0[keep], rtol=1e-12 if precision == "fp64" else 2e-6)
    h.close()


def test_closed_ternary_tube_fp64():
    """The ternary tube of Sec. 4.2 closed by walls (the paper's Loschmidt
    setting), 300 steps, against the oracle."""
    wl = W.ternary_tube(steps=300)
    prm = oracle_params(wl, walls_x=True)
    ref = O.run(O.init_populations(wl.X, wl.u, wl.T, wl.P, prm), prm, wl.steps)
    h = gpu_handle(wl, "fp64", walls_x=True)
    h.init_fields(wl.X, wl.u, wl.T, wl.P)
    h.step(wl.steps)
    assert rel(h.populations(), ref) < TOL["fp64"]
    errs = field_errors(h.moments_dict(), _moments(ref, prm), _cs(wl))
    assert max(errs.values()) < TOL["fp64"], errs
    h.close()
