"""A small, fixed case of the step for profilers: build the library, set up
one workload, run a few steps and exit.

    python -m paper_2004_11286_gb300.profile_case fp32 96 shear [steps]

Arguments: storage precision (fp64, fp32, fp16, bf16), grid edge, workload
(``shear``: the two-component shear layer; ``acoustic``: the binary
pressure pulse; ``mixture``: the 8-species smooth mixture) and the step count
(default 4, so that one collide of each streaming parity runs after the
first)."""

from __future__ import annotations

import sys


def main(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    from paper_2004_11286_gb300 import binding, build, workloads as W
    build.build()
    prec = argv[0] if argv else "fp32"
    n = int(argv[1]) if len(argv) > 1 else 96
    name = argv[2] if len(argv) > 2 else "acoustic"
    steps = int(argv[3]) if len(argv) > 3 else 4
    if name == "acoustic":
        wl = W.acoustic_pulse(n=n, sigma=6.0 * n / 128)
    elif name == "shear":
        wl = W.shear_layer(n=n)
    elif name == "mixture":
        wl = W.random_mixture(M=8, n=n)
    else:
        raise SystemExit(f"unknown workload {name!r}")
    h = binding.from_workload(wl, precision=prec, slaved=W.slaved_species(wl))
    h.init_fields(wl.X, wl.u, wl.T, wl.P)
    h.step(steps)
    h.synchronize()
    h.close()
    print("ok", prec, name, n, steps)


if __name__ == "__main__":
    main()
