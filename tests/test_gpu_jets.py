"""The opposed jets of Sec. 4.3 on the GPU: the boundary set (equilibrium
inlets, free-slip walls, zero-gradient outlets) on a frame of outside nodes
around the domain (include/lbm_mix.h, LBM_BC_JET / LBM_BC_OUTLET).

  * parity with the FP64 oracle's boundary set (oracle.Frame) on the domain's
    interior: FP64 to 1e-12 and FP32 to 1e-5 on the populations, over both
    streaming parities and 40 steps, in two and three dimensions;
  * the host's refusals of unsupported combinations;
  * the paper's 200 x 400 x 1 case run to a steady stagnation flow: the jets
    meet near the middle, and hydrogen and water from the left jet diffuse
    against the bulk flow into the right jet's side of the stagnation plane
    (the case's point: diffusion opposed by the flow; hydrogen, the fastest
    diffuser, far more than water)."""

import types

import numpy as np
import pytest

import oracle as O
from paper_2004_11286_gb300 import workloads as W

from gpu_helpers import TOL, gpu_handle, oracle_params, rel

pytestmark = pytest.mark.gpu


def _inlet_pops(wl, inl, prm):
    """Complete equilibrium populations (S, 27) of the two inlet states."""
    out = []
    for k in range(2):
        u = np.array([[inl.u[k]], [0.0], [0.0]])
        out.append(O.init_populations(inl.X[k][:, None], u, np.array([inl.T[k]]), np.array([inl.P[k]]), prm)[..., 0])
    return tuple(out)


def _grid_jets(inl):
    """The nozzles in grid rows (the frame adds one row below the interior)."""
    return types.SimpleNamespace(y0=inl.y0 + 1, y1=inl.y1 + 1, X=inl.X, u=inl.u, T=inl.T, P=inl.P)


def _setup(shape, U=0.02, seed=0):
    nz, ny, nx = shape
    wl, inl = W.opposed_jets(nx=nx, ny=ny, nz=nz, U=U, nozzle=(0.25, 0.75))
    prm0 = oracle_params(wl)
    fr = O.Frame(y0=inl.y0, y1=inl.y1, inlet=_inlet_pops(wl, inl, prm0))
    prm = oracle_params(wl, frame=fr)
    return wl, inl, prm


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(1, 16, 12), (3, 10, 8)])
def test_jets_match_the_oracle(shape, precision):
    wl, inl, prm = _setup(shape)
    pops = O.init_populations(wl.X, wl.u, wl.T, wl.P, prm)
    h = gpu_handle(W.Workload(wl.name, wl.molar_mass, wl.cv_molar, wl.D, wl.mu, wl.lam, W.with_frame(wl.X),
                              W.with_frame(wl.u), W.with_frame(wl.T), W.with_frame(wl.P), wl.steps),
                   precision, jets=_grid_jets(inl))
    h.init_fields(W.with_frame(wl.X), W.with_frame(wl.u), W.with_frame(wl.T), W.with_frame(wl.P))
    ref = pops
    worst = 0.0
    for s in range(1, 41):
        ref = O.step(ref, prm)
        h.step(1)
        if s in (1, 2, 3, 10, 25, 40):
            got = h.populations()[..., 1:-1, 1:-1]
            e = rel(got, ref)
            worst = max(worst, e)
            assert e < TOL[precision], (s, e)
    mac = O.macroscopic(ref, prm)
    gm = h.moments_dict()
    assert rel(gm["u"][..., 1:-1, 1:-1], mac["u"]) < (1e-10 if precision == "fp64" else 1e-4)
    assert np.abs(mac["u"][0][..., 0]).max() > 1e-3            # the jets are flowing
    h.close()
    print(shape, precision, f"worst population error {worst:.2e}")


def test_jets_refusals():
    from paper_2004_11286_gb300 import binding
    wl, inl, _ = _setup((1, 8, 8))
    args = (wl.molar_mass, wl.cv_molar, wl.D)
    kw = dict(mu=wl.mu, lam=wl.lam, shape=(1, 10, 10), jets=_grid_jets(inl))
    for bad in (dict(precision="bf16"), dict(precision="fp32", closure="mlp"),
                dict(precision="fp32", cv_poly=np.tile([[2.5]], (wl.M, 1)))):
        with pytest.raises(binding.LbmError) as e:
            binding.LbmMix(*args, **{**kw, **bad})
        assert "UNSUPPORTED" in str(e.value)
    bad_rows = types.SimpleNamespace(**{**vars(_grid_jets(inl)), "y0": 0})
    with pytest.raises(binding.LbmError) as e:
        binding.LbmMix(*args, **{**kw, "jets": bad_rows, "precision": "fp32"})
    assert "ERR_ARG" in str(e.value)


def test_paper_jets_reach_a_stagnation_flow():
    """200 x 400 x 1, nozzles over [0.1, 0.9] of the height, FP32, run until
    the fields stop changing.  On the stagnation line (mid-height) u_x
    changes sign once, near the middle, and hydrogen and water, fed only by
    the left jet, reach the right of the stagnation point at mole fractions
    above the right jet's floor: diffusion against the bulk flow."""
    wl, inl = W.opposed_jets()
    h = gpu_handle(W.Workload(wl.name, wl.molar_mass, wl.cv_molar, wl.D, wl.mu, wl.lam, W.with_frame(wl.X),
                              W.with_frame(wl.u), W.with_frame(wl.T), W.with_frame(wl.P), wl.steps),
                   "fp32", jets=_grid_jets(inl))
    h.init_fields(W.with_frame(wl.X), W.with_frame(wl.u), W.with_frame(wl.T), W.with_frame(wl.P))
    prev = None
    for _ in range(10):
        h.step(4000)
        m = h.moments_dict()
        line = m["X"][:, 0, 201, 1:-1].copy()
        if prev is not None:
            change = np.abs(line - prev).max()
        prev = line
    ux = m["u"][0, 0, 201, 1:-1]
    assert np.isfinite(m["u"]).all()
    sign_changes = np.nonzero(np.diff(np.sign(ux)))[0]
    assert len(sign_changes) == 1
    xs = int(sign_changes[0])
    assert 60 < xs < 140, xs
    h2, h2o = line[0], line[3]
    floor_h2, floor_h2o = inl.X[1][0], inl.X[1][3]
    right = slice(xs + 5, xs + 15)
    print("stagnation point", xs, "H2 right of it", h2[right].round(4), "H2O right of it", h2o[right].round(4),
          "change over the last 4000 steps", f"{change:.1e}")
    assert (h2[right] > 1.5 * floor_h2).all()
    assert (h2o[right] > 1.02 * floor_h2o).all()
    h.close()
