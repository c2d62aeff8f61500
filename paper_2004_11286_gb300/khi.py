"""The three-dimensional Kelvin-Helmholtz flow of Sec. 4.5 (N2 / H2O), run
on the GPU with the turbulent kinetic energy spectrum and mixing diagnostics
along the way.

    python -m paper_2004_11286_gb300.khi --shape 200x800x800 --steps 200
    python -m paper_2004_11286_gb300.khi --shape 64x256x256 --te 8 --every 1

--shape is Lz x Ly x Lx.  The Reynolds number is the paper's (11963.46 on
its 800-cell layer) scaled with Ly, so every box runs at the paper's lattice
viscosity (the full box at exactly its Re).  Time is counted in eddy
turnover times t_e = Lx / U_r (U_r the initial relative velocity).  Prints
one JSON document: per output time the spectrum, its slope over the fit
range, the fluctuating kinetic energy, the mixing-layer thickness, the
temperature range and the conservation sums."""

from __future__ import annotations

import argparse
import json
import time

import numpy as np


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--shape", default="64x256x256")
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--te", type=float, default=0.0, help="run to this many eddy turnover times")
    ap.add_argument("--steps", type=int, default=0, help="or this many steps")
    ap.add_argument("--every", type=float, default=1.0, help="output every this many t_e")
    ap.add_argument("--fit", nargs=2, type=float, default=None, metavar=("KMIN", "KMAX"),
                    help="slope fit range in units of 2 pi / Lmax (default Lmax/32 .. Lmax/8)")
    ap.add_argument("--out", default=None)
    return ap.parse_args()


def run(shape, precision="fp32", te=0.0, steps=0, every=1.0, fit=None):
    import torch
    from paper_2004_11286_gb300 import binding, workloads as W
    from paper_2004_11286_gb300.diagnostics import spectral_slope, tke_spectrum
    nz, ny, nx = shape
    wl = W.khi_n2_h2o(shape=shape, reynolds=11963.46 * ny / 800.0)
    Ur = 2.0 * float(np.abs(wl.u[0]).max())
    t_e = nx / Ur
    total = steps if steps > 0 else int(round(te * t_e))
    chunk = max(1, int(round(every * t_e))) if te > 0 else total
    L = max(shape)
    kmin, kmax = fit if fit is not None else (L / 32.0, L / 8.0)
    h = binding.from_workload(wl, precision=precision, slaved=W.slaved_species(wl))
    h.init_fields(wl.X, wl.u, wl.T, wl.P)
    s0 = h.diagnostics()
    out = {"shape": list(shape), "precision": precision, "reynolds": 11963.46 * ny / 800.0,
           "t_e_steps": t_e, "U_r": Ur, "fit_range": [kmin, kmax], "outputs": []}
    cons = [wl.M, wl.M + 4]          # mixture mass and total energy
    done, busy = 0, 0.0
    while done < total:
        n = min(chunk, total - done)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.step(n)
        h.synchronize()
        busy += time.perf_counter() - t0
        done += n
        m = h.moments_dict()
        k, E = tke_spectrum(m["u"], m["rho"])
        xn2 = m["X"][0].mean(axis=(0, 2))
        s = h.diagnostics()
        out["outputs"].append({
            "step": done, "t_e": done / t_e,
            "slope": spectral_slope(k, E, kmin, kmax) if E[1:].sum() > 0 else None,
            "k": [float(v) for v in k[: L // 2]], "E": [float(v) for v in E[: L // 2]],
            "tke": float(E.sum()),
            "mixing_thickness": float(((xn2 > 0.2) & (xn2 < 0.8)).sum()),
            "T_range": [float(m["T"].min()), float(m["T"].max())],
            "conservation_rel": float(np.max(np.abs(s - s0)[cons] / np.abs(s0)[cons])),
            "finite": bool(np.isfinite(m["u"]).all())})
    out["mlups"] = wl.nodes * total / busy / 1e6
    h.close()
    return out


def main():
    a = _args()
    shape = tuple(int(v) for v in a.shape.split("x"))
    res = run(shape, a.precision, a.te, a.steps, a.every, a.fit)
    txt = json.dumps(res)
    if a.out:
        with open(a.out, "w") as f:
            f.write(txt)
    brief = {k: v for k, v in res.items() if k != "outputs"}
    brief["outputs"] = [{k: v for k, v in o.items() if k not in ("k", "E")} for o in res["outputs"]]
    print(json.dumps(brief))


if __name__ == "__main__":
    main()
