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
    """Relative errors per observable, max |a - b| / max(||b||_inf, floor):
    rho, T, P unfloored; velocity floored at 1e-3 c_s (u = j / rho is the
    small difference of populations of size rho w_i, so where the fluid is
    nearly at rest its attainable relative accuracy degrades as c_s / |u|);
    mole fractions absolutely (X_a ~ 0 in places)."""
    return dict(rho=rel(gm["rho"], om["rho"]), T=rel(gm["T"], om["T"]), P=rel(gm["P"], om["P"]),
                u=rel(gm["u"], om["u"], floor=1e-3 * cs),
                X=float(np.abs(gm["X"] - om["X"]).max()))


def deviation_errors(gm, om, min_signal=1e-4):
    """Errors of the fields' deviations from their domain means, relative to
    the oracle's deviation: max |(a - mean a) - (b - mean b)| / max |b - mean b|,
    for rho, T, P and each X_a whose oracle deviation is live (at least
    ``min_signal`` of the field's magnitude); the plain relative error of a
    field that varies by 1e-4 can hide an error as large as its variation."""
    out = {}
    for k in ("rho", "T", "P"):
        a, b = np.asarray(gm[k]), np.asarray(om[k])
        db = b - b.mean()
        den = float(np.abs(db).max())
        if den >= min_signal * float(np.abs(b).max()):
            out[k] = float(np.abs((a - a.mean()) - db).max() / den)
    Xa, Xb = np.asarray(gm["X"]), np.asarray(om["X"])
    for s in range(Xb.shape[0]):
        db = Xb[s] - Xb[s].mean()
        den = float(np.abs(db).max())
        if den >= min_signal:
            out[f"X{s}"] = float(np.abs((Xa[s] - Xa[s].mean()) - db).max() / den)
    return out
