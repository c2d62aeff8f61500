"""Pins of the oracle's opposed-jets boundary set (Sec. 4.3; the readings
are in the oracle's docstring): free-slip walls, zero-gradient outlets and
equilibrium inlets, each checked against a property that the boundary rule
must have and that the periodic oracle fixes independently."""

import numpy as np
import pytest

import oracle as O
from paper_2004_11286_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _params(wl, frame=None, **kw):
    return O.Params(wl.molar_mass, wl.cv_molar, wl.D, mu=wl.mu, lam=wl.lam, slaved=W.slaved_species(wl),
                    frame=frame, **kw)


def _random_state(shape, seed, velocity=0.02):
    wl = W.random_mixture(M=3, shape=shape, seed=seed, velocity=velocity, amplitude=0.3)
    return wl


def test_free_slip_walls_are_a_mirror_plane():
    """Specular reflection halfway between the boundary node and the outside
    node makes each x wall a mirror plane.  With free-slip walls on both x
    faces (no nozzle) and y, z periodic, any state evolves exactly as the left
    half of the periodic domain of twice the width holding the state and its
    mirror image (x velocities reflected).  This pins the reflected
    populations and the mirror rule of the derivative (Phi_x odd, the rest
    even)."""
    wl = _random_state((3, 4, 5), seed=31)
    fr = O.Frame(y0=0, y1=0, inlet=(), x_faces=True, y_faces=False)
    prm = _params(wl, fr)
    pops = O.init_populations(wl.X, wl.u, wl.T, wl.P, prm) * W.perturbation((prm.S, 27) + wl.shape, 0.01, 5)
    nx = wl.shape[-1]
    big = np.concatenate([pops, pops[:, O.XREF][..., ::-1]], axis=-1)
    prm_big = _params(wl)
    a, b = pops, big
    for _ in range(6):
        a = O.step(a, prm)
        b = O.step(b, prm_big)
    assert np.abs(a - b[..., :nx]).max() < 1e-13 * np.abs(b).max()
    # the right half stays the mirror image (a check of the reference itself)
    assert np.abs(b[..., nx:] - b[:, O.XREF][..., :nx][..., ::-1]).max() < 1e-13 * np.abs(b).max()


@pytest.mark.parametrize("uy", [0.0, 0.03])
def test_outlets_pass_a_flow_uniform_along_them(uy):
    """A zero-normal-gradient outlet leaves a state that does not vary
    across it unchanged: with outlets on both y faces and x, z periodic, a
    state uniform in y (here also leaving through the outlets at velocity uy)
    evolves exactly as on the y-periodic grid."""
    wl = _random_state((3, 4, 6), seed=32)
    for a in range(wl.M):
        wl.X[a] = wl.X[a][:, :1, :]
    wl.u[:] = wl.u[:, :, :1, :]
    wl.u[1] = uy
    fr = O.Frame(y0=0, y1=0, inlet=(), x_faces=False, y_faces=True)
    prm, prm_per = _params(wl, fr), _params(wl)
    pops = O.init_populations(wl.X, wl.u, wl.T, wl.P, prm)
    a, b = pops, pops
    for _ in range(5):
        a = O.step(a, prm)
        b = O.step(b, prm_per)
    assert np.abs(a - b).max() < 1e-13 * np.abs(b).max()
    assert np.abs(np.diff(a, axis=-2)).max() < 1e-13 * np.abs(a).max()


def test_inlets_hold_a_uniform_flow():
    """Inlets that feed the equilibrium of the interior's own uniform moving
    state keep it exactly: with nozzles over the whole of both x faces, y
    and z periodic, the uniform flow at u = (U, 0, 0) is a fixed point."""
    wl = _random_state((2, 3, 6), seed=33, velocity=0.0)
    Xu = np.array([0.2, 0.5, 0.3])
    wl.X[:] = Xu[:, None, None, None]
    wl.u[:] = 0.0
    wl.u[0] = 0.02
    prm0 = _params(wl)
    inlet = O.init_populations(Xu[:, None], np.array([[0.02], [0.0], [0.0]]), np.array([wl.T.flat[0]]),
                               np.array([wl.P.flat[0]]), prm0)[..., 0]
    fr = O.Frame(y0=0, y1=wl.shape[1], inlet=(inlet, inlet), x_faces=True, y_faces=False)
    prm = _params(wl, fr)
    pops = O.init_populations(wl.X, wl.u, wl.T, wl.P, prm)
    a = pops
    for _ in range(5):
        a = O.step(a, prm)
    assert np.abs(a - pops).max() < 1e-14 * np.abs(pops).max()


def test_symmetric_jets_stay_symmetric():
    """Two jets of the same composition meeting head on, each at speed U, in
    a box whose nozzles and outlets are placed symmetrically: the flow keeps
    both mirror symmetries (left-right with x velocities reflected, up-down
    with y velocities reflected).  Each face's rule is written separately,
    so a mistake on one side breaks the symmetry."""
    wl, inl = W.opposed_jets(nx=8, ny=10, nz=1, U=0.02)
    Xs = inl.X[0]
    wl.X[:] = Xs[:, None, None, None]
    prm0 = _params(wl)
    T0, P0 = wl.T.flat[0], wl.P.flat[0]
    eq = lambda ux: O.init_populations(Xs[:, None], np.array([[ux], [0.0], [0.0]]), np.array([T0]),
                                       np.array([P0]), prm0)[..., 0]
    fr = O.Frame(y0=inl.y0, y1=inl.y1, inlet=(eq(0.02), eq(-0.02)))
    prm = _params(wl, fr)
    a = O.init_populations(wl.X, wl.u, wl.T, wl.P, prm)
    YREF = np.array([int(np.where((O.C == O.C[i] * np.array([1, -1, 1])).all(axis=1))[0][0]) for i in range(27)])
    for _ in range(20):
        a = O.step(a, prm)
    scale = np.abs(a).max()
    assert np.abs(a - a[:, O.XREF][..., ::-1]).max() < 1e-13 * scale
    assert np.abs(a - a[:, YREF][..., ::-1, :]).max() < 1e-13 * scale
    mac = O.macroscopic(a, prm)
    ux = mac["u"][0, 0]
    assert ux[:, 0].mean() > 0.0 and ux[:, -1].mean() < 0.0      # the jets flow in
    uy = mac["u"][1, 0]
    assert uy[0, :].mean() < 0.0 and uy[-1, :].mean() > 0.0      # and leave through the outlets


def test_frame_derivative_closed_forms():
    """The derivative beyond the frame, in closed form on fields whose
    continuation is known.  Outlets and nozzles (nearest-value rule): a field
    of slope 1 across the face has derivative 1/2 on the boundary row (the
    stencil's one-sided mean).  Free-slip walls (mirror rule): x + 1/2 is odd
    and (x + 1/2)^2 even about the wall at x = -1/2, so their mirror images
    continue them exactly and the derivative is the interior one, 1."""
    nz, ny, nx = 2, 8, 5
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    fr = O.Frame(y0=2, y1=6, inlet=(), x_faces=True, y_faces=True)
    dy = O.iso_derivative(y.astype(float), 1, frame=fr)
    assert np.allclose(dy[:, 1:-1], 1.0, atol=1e-14)
    assert np.allclose(dy[:, 0], 0.5, atol=1e-14) and np.allclose(dy[:, -1], 0.5, atol=1e-14)
    odd = x + 0.5
    d_odd = O.iso_derivative(odd, 0, odd_x=True, frame=fr)
    # rows whose three outside neighbours all lie on a wall, or all in a nozzle
    walls, nozzles = [0, ny - 1], [fr.y0 + 1, fr.y1 - 2]
    assert np.allclose(d_odd[:, walls, 0], 1.0, atol=1e-14)       # mirror (odd) at the walls
    assert np.allclose(d_odd[:, nozzles, 0], 0.5, atol=1e-14)     # nearest value at the nozzles
    even = (x + 0.5) ** 2
    d_even = O.iso_derivative(even, 0, frame=fr)
    assert np.allclose(d_even[:, :, 0], 1.0, atol=1e-13)          # 2 (x + 1/2) at x = 0, any row
    mirror_right = (nx - 0.5 - x) ** 2                             # even about x = nx - 1/2
    assert np.allclose(O.iso_derivative(mirror_right, 0, frame=fr)[:, :, -1], -1.0, atol=1e-13)


def test_outlets_let_a_composition_bump_leave():
    """A composition bump carried up by a uniform flow leaves through the
    outlet: the species' total mass falls, where on the y-periodic grid the
    same bump re-enters at the bottom and the mass is conserved exactly."""
    wl = _random_state((1, 12, 3), seed=34, velocity=0.0)
    ny = wl.shape[1]
    yy = np.arange(ny)[None, None, :, None]
    bump = np.broadcast_to(0.2 * np.exp(-0.5 * ((yy[0] - (ny - 2.0)) / 1.5) ** 2), wl.shape)
    X = np.stack([0.3 + bump, 0.4 - bump, np.full(wl.shape, 0.3)])
    wl.X[:] = X / X.sum(axis=0, keepdims=True)
    wl.u[:] = 0.0
    wl.u[1] = 0.05
    fr = O.Frame(y0=0, y1=0, inlet=(), x_faces=False, y_faces=True)
    prm, prm_per = _params(wl, fr), _params(wl)
    pops = O.init_populations(wl.X, wl.u, wl.T, wl.P, prm)
    mass = lambda p: p[0].sum()
    a, b = pops, pops
    for _ in range(30):
        a = O.step(a, prm)
        b = O.step(b, prm_per)
    assert abs(mass(b) - mass(pops)) < 1e-12 * mass(pops)
    assert mass(a) < mass(pops) * (1.0 - 1e-3)


def test_jets_recipe():
    """The opposed-jets inputs: the printed jet compositions (floored and
    renormalised), nozzles over [0.1, 0.9] of the height, jets of equal
    momentum flux rho U^2 at a common T and P, and the framed grid one node
    larger on every x and y face."""
    wl, inl = W.opposed_jets()
    assert wl.shape == (1, 400, 200)
    assert (inl.y0, inl.y1) == (40, 360)
    for k in range(2):
        assert abs(inl.X[k].sum() - 1.0) < 1e-15 and inl.X[k].min() > 0.0098   # floor 0.01, renormalised
    assert inl.X[0][0] > 0.09 and inl.X[1][2] > 0.09             # H2 left, O2 right, as printed
    rho = [float(inl.X[k] @ wl.molar_mass) * inl.P[k] / inl.T[k] for k in range(2)]
    assert inl.u[0] > 0 > inl.u[1]
    assert abs(rho[0] * inl.u[0] ** 2 - rho[1] * inl.u[1] ** 2) < 1e-12 * rho[0] * inl.u[0] ** 2
    framed = W.with_frame(wl.X)
    assert framed.shape == (wl.M, 1, 402, 202)
    assert np.array_equal(framed[..., 1:-1, 1:-1], wl.X)
    assert np.array_equal(framed[..., 0, 1:-1], wl.X[..., 0, :])
