"""Pins of the oracle's bounce-back walls (the closed tube of Sec. 4.2,
walls normal to x), no GPU.

* Mirror equivalence: for a state that varies along x only, with no y or z
  velocity, bounce-back reverses a population exactly as a mirror would, and
  the derivative's wall rule is the mirror image.  The walled tube of width
  nx must therefore evolve exactly as the left half of the periodic tube of
  width 2 nx that holds the state and its mirror image (u_x odd, everything
  else even).  A wrong sign in the Phi_x rule, a shifted reflected
  population or a wrong wall node fails this.
* A closed box conserves the mass of every unslaved species, the mixture
  mass and the total energy (each population either streams to a neighbour
  or returns to its node).
* A resting uniform mixture stays at rest (the rest equilibrium is symmetric
  under c -> -c, so reflected populations are what a neighbour would send).
"""

import numpy as np
import pytest

import oracle as O


def _params(M=3, walls=True, coupling="strong"):
    mm = np.array([2.0, 40.0, 16.0, 28.0][:M])
    cv = np.array([2.5, 1.5, 3.0, 2.5][:M])
    D = np.array([[0.0, 0.05, 0.05, 0.02], [0.05, 0.0, 0.01, 0.03],
                  [0.05, 0.01, 0.0, 0.04], [0.02, 0.03, 0.04, 0.0]])[:M, :M]
    P0 = 0.2 / float(mm.mean())
    mu = np.full(M, 0.1 * P0)
    lam = mu * (cv + 1.0) / mm / 0.71
    return O.Params(mm, cv, D, mu=mu, lam=lam, coupling=coupling, slaved=1, walls_x=walls)


def _fields_x(M, nx, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.arange(nx)
    X = np.empty((M, 1, 1, nx))
    for a in range(M):
        X[a, 0, 0] = 1.0 + 0.4 * np.sin(2 * np.pi * (x + rng.uniform()) / nx * (a + 1))
    X /= X.sum(axis=0)
    u = np.zeros((3, 1, 1, nx))
    u[0, 0, 0] = 0.02 * np.sin(np.pi * (x + 0.5) / nx) * rng.uniform(0.5, 1.0)
    T = 0.2 * (1.0 + 0.05 * np.cos(2 * np.pi * x / nx))[None, None, :]
    P = (0.2 / 20.0) * (1.0 + 0.02 * np.cos(np.pi * x / nx))[None, None, :]
    return X, u, T, P


def _mirror(a, odd=False):
    m = a[..., ::-1]
    return np.concatenate([a, -m if odd else m], axis=-1)


@pytest.mark.parametrize("coupling", ["strong", "weak"])
def test_walled_tube_equals_mirrored_periodic_tube(coupling):
    M, nx, steps = 3, 6, 25
    X, u, T, P = _fields_x(M, nx, 5)
    pw = _params(M, True, coupling)
    pp = _params(M, False, coupling)
    walled = O.run(O.init_populations(X, u, T, P, pw), pw, steps)
    Xm = _mirror(X)
    um = np.stack([_mirror(u[0], odd=True), _mirror(u[1]), _mirror(u[2])])
    per = O.run(O.init_populations(Xm, um, _mirror(T), _mirror(P), pp), pp, steps)
    scale = np.abs(walled).max()
    assert np.abs(per[..., :nx] - walled).max() < 1e-13 * scale
    # the walls did something: the periodic tube of width nx differs
    per_nx = O.run(O.init_populations(X, u, T, P, pp), pp, steps)
    assert np.abs(per_nx - walled).max() > 1e-6 * scale


def test_closed_box_conserves_mass_and_energy():
    prm = _params(3, True)
    rng = np.random.Generator(np.random.PCG64(9))
    shape = (3, 4, 5)
    X = rng.uniform(0.3, 1.0, (3,) + shape)
    X /= X.sum(axis=0)
    u = rng.uniform(-0.02, 0.02, (3,) + shape)
    T = 0.2 * (1.0 + rng.uniform(-0.03, 0.03, shape))
    P = (0.2 / 20.0) * (1.0 + rng.uniform(-0.02, 0.02, shape))
    pops = O.init_populations(X, u, T, P, prm)
    s0 = O.conserved_sums(pops, prm)
    pops = O.run(pops, prm, 30)
    s1 = O.conserved_sums(pops, prm)
    # every species but the slaved one (its populations relax to the
    # mixture's deficit, Eq. rhoMATCH), the mixture density and rho E
    keep = [a for a in range(prm.M) if a != prm.slaved] + [prm.M, prm.M + 4]
    for k in keep:
        assert abs(s1[k] - s0[k]) < 1e-13 * abs(s0[k]), k
    # the walls exchange momentum with the fluid: the x momentum changes
    assert abs(s1[prm.M + 1] - s0[prm.M + 1]) > 1e-12 * abs(s0[prm.M])


def test_resting_mixture_stays_at_rest():
    prm = _params(3, True)
    shape = (2, 3, 4)
    X = np.stack([np.full(shape, v) for v in (0.5, 0.3, 0.2)])
    pops = O.init_populations(X, np.zeros((3,) + shape), np.full(shape, 0.2), np.full(shape, 0.01), prm)
    out = O.run(pops, prm, 5)
    # the walls are invisible: the same steps on the periodic box give the
    # same populations, bit for bit, and both stay at rest to rounding
    per = O.run(pops, _params(3, False), 5)
    np.testing.assert_array_equal(out, per)
    assert np.abs(out - pops).max() < 1e-13 * np.abs(pops).max()


def test_stream_reflects_at_the_walls_only():
    rng = np.random.Generator(np.random.PCG64(3))
    post = rng.uniform(size=(2, 27, 2, 3, 4))
    out = O.stream(post, walls_x=True)
    ref = O.stream(post)
    for i in range(27):
        cx = O.C[i, 0]
        inner = slice(1, 4) if cx > 0 else (slice(0, 3) if cx < 0 else slice(0, 4))
        np.testing.assert_array_equal(out[:, i, :, :, inner], ref[:, i, :, :, inner])
        if cx > 0:
            np.testing.assert_array_equal(out[:, i, :, :, 0], post[:, O.OPP[i], :, :, 0])
        if cx < 0:
            np.testing.assert_array_equal(out[:, i, :, :, 3], post[:, O.OPP[i], :, :, 3])
    # every value is moved, not created: per-lattice sums are unchanged
    np.testing.assert_allclose(out.sum(axis=(1, 2, 3, 4)), post.sum(axis=(1, 2, 3, 4)), rtol=1e-14)
