"""Physics of the GPU step at the benchmark's full size, independent of the
oracle: the speed of sound of the binary acoustic pulse (128^3, m = 4, 40,
FP32) for mole fractions 0.2, 0.5 and 0.8 against the mixture's ideal-gas
closed form sqrt(gamma R T) (Secs. 4.1, 4.4, Eq. soundSpeed)."""

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


@pytest.mark.parametrize("x1", [0.2, 0.5, 0.8])
def test_acoustic_pulse_speed_of_sound(x1):
    """Along the +x axis r (P - P0) of the outgoing spherical wave keeps the
    shape of a 1-D pulse moving at c (the 1/r of the spherical solution is
    divided out), so its maximum travels at the speed of sound."""
    wl = W.acoustic_pulse(x1=x1)
    n = wl.shape[2]
    c = n // 2
    P0 = float(wl.P.min())
    h = gpu_handle(wl, "fp32")
    h.init_fields(wl.X, wl.u, wl.T, wl.P)
    times, pos = [], []
    t = 0
    for target in range(60, 200, 20):
        h.step(target - t)
        t = target
        P = h.moments_dict()["P"][c, c, c:]
        r = np.arange(P.size, dtype=float)
        q = r * (P - P0)
        k = int(np.argmax(q[5:-5])) + 5
        a, b, d = q[k - 1], q[k], q[k + 1]
        pos.append(k + 0.5 * (a - d) / (a - 2 * b + d))     # parabolic peak
        times.append(t)
    h.close()
    c_meas = np.polyfit(times, pos, 1)[0]
    cs, c_iso = _closed_form(wl)
    assert abs(c_meas / cs - 1.0) < 0.02, (x1, c_meas, cs)
    assert abs(c_meas / c_iso - 1.0) > 0.1          # the adiabatic, not the isothermal speed
