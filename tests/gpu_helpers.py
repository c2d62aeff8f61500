"""Shared helpers of the GPU parity tests (not a test module)."""

import numpy as np

import oracle as O
from paper_2004_11286_gb300 import workloads as W

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def oracle_params(wl, coupling="strong", slaved=None, **kw):
    return O.Params(wl.molar_mass, wl.cv_molar, wl.D, mu=wl.mu, lam=wl.lam, R_U=wl.R_U,
                    coupling=coupling, slaved=W.slaved_species(wl) if slaved is None else slaved, **kw)


def gpu_handle(wl, precision, coupling="strong", slaved=None, **kw):
    from paper_2004_11286_gb300 import binding
    return binding.LbmMix(wl.molar_mass, wl.cv_molar, wl.D, mu=wl.mu, lam=wl.lam, shape=wl.shape,
                          precision=precision, coupling=coupling, R_U=wl.R_U,
                          slaved=W.slaved_species(wl) if slaved is None else slaved, **kw)


def rel(a, b, floor=0.0):
    """max |a - b| / max(||b||_inf, floor)."""
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(float(np.abs(b).max()), floor))


def field_errors(gm, om, cs):
    """Relative errors per observable.  Velocity is floored at 1e-2 c_s: u =
    j / rho is the small difference of populations of size rho w_i, so its
    attainable relative accuracy degrades as c_s / |u|.  Mole fractions are
    compared absolutely."""
    return dict(rho=rel(gm["rho"], om["rho"]), T=rel(gm["T"], om["T"]), P=rel(gm["P"], om["P"]),
                u=rel(gm["u"], om["u"], floor=1e-2 * cs),
                X=float(np.abs(gm["X"] - om["X"]).max()))
