"""Pins of the FP64 oracle against what the paper and the mathematics fix
(no GPU).  Each test names the passage it checks; together they are chosen so
that a dropped term, a wrong sign or index, or a transposed operand anywhere
in the oracle fails at least one of them."""

import os

import numpy as np
import pytest

import oracle as O

RNG = np.random.Generator(np.random.PCG64(20040)).uniform
HERE = os.path.dirname(os.path.abspath(__file__))


def _rand_params(M, coupling="strong", seed=0, fixed=False):
    rng = np.random.Generator(np.random.PCG64(seed))
    mm = rng.uniform(2.0, 44.0, M)
    cv = rng.choice([1.5, 2.5, 3.0], M)
    D = np.zeros((M, M))
    for a in range(M):
        for b in range(a + 1, M):
            D[a, b] = D[b, a] = np.exp(rng.uniform(np.log(0.005), np.log(0.1)))
    if M == 1:
        D[0, 0] = 0.05
    kw = dict(omega_fixed=1.6, omega1_fixed=1.2) if fixed else dict(
        mu=rng.uniform(0.002, 0.004, M), lam=rng.uniform(0.004, 0.02, M))
    # slave the species carrying most mass (Sec. 3.5.2 advice), so the slaved
    # density stays positive under the random perturbations below
    return O.Params(mm, cv, D, coupling=coupling, slaved=int(np.argmax(mm)), **kw)


def _rand_state(prm, shape, seed=1, du=0.05, noise=0.02):
    """Random smooth-ish equilibrium fields, then perturbed populations."""
    rng = np.random.Generator(np.random.PCG64(seed))
    M = prm.M
    X = rng.uniform(0.2, 1.0, (M,) + shape)
    X /= X.sum(axis=0)
    u = rng.uniform(-du, du, (3,) + shape)
    T = rng.uniform(0.4, 0.6, shape)
    P = rng.uniform(0.02, 0.03, shape)
    pops = O.init_populations(X, u, T, P, prm)
    pops = pops * (1.0 + noise * rng.uniform(-1, 1, pops.shape))
    return pops


# ---------------------------------------------------------------------------
# Sec. 2.4, Eq. (prod): product-form moments
# ---------------------------------------------------------------------------
def test_psi_product_moments():
    C = O.C.astype(float)
    for _ in range(5):
        xi = RNG(-0.3, 0.3, 3)
        zeta = RNG(0.05, 0.6)
        psi = O.psi_product(xi, np.array(zeta))
        assert np.isclose(psi.sum(), 1.0, atol=1e-15)
        np.testing.assert_allclose(psi @ C, xi, atol=1e-15)
        second = np.einsum("i,ia,ib->ab", psi, C, C)
        np.testing.assert_allclose(second, zeta * np.eye(3) + np.outer(xi, xi), atol=1e-15)
        # lattice constraint c^3 = c: diagonal third moment equals xi (the
        # defect corrected by Eq. fwithcorrection); off-diagonal ones factor.
        np.testing.assert_allclose(np.einsum("i,ia->a", psi, C ** 3), xi, atol=1e-15)
        assert np.isclose(np.einsum("i,i,i,i", psi, C[:, 0], C[:, 1], C[:, 2]), xi.prod(), atol=1e-15)
        assert np.isclose(np.einsum("i,i,i", psi, C[:, 0] ** 2, C[:, 1]), (zeta + xi[0] ** 2) * xi[1],
                          atol=1e-15)


# ---------------------------------------------------------------------------
# Sec. 3.4.1: the ansatz reproduces {M0, m, M} for any theta
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("theta", [0.02, 0.1, 1.0 / 3.0, 0.5, 0.9])
def test_g_ansatz_moments(theta):
    C = O.C.astype(float)
    M0 = RNG(0.5, 2.0)
    m = RNG(-0.2, 0.2, 3)
    A = RNG(-0.1, 0.1, (3, 3))
    Mt = A + A.T + np.eye(3) * RNG(0.2, 0.8)
    G = O.g_ansatz(np.array(theta), np.array(M0), m, Mt)
    assert np.isclose(G.sum(), M0, rtol=1e-14)
    np.testing.assert_allclose(G @ C, m, atol=1e-14)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", G, C, C), Mt, atol=1e-13)


def test_g_ansatz_is_grad_at_reference_temperature():
    """At theta = 1/3 the Z-correction vanishes (Sec. 3.4.1): G equals the
    second-order Hermite (Grad) expansion with the D3Q27 weights 8/27, 2/27,
    1/54, 1/216."""
    C = O.C.astype(float)
    th = 1.0 / 3.0
    M0, m = 1.3, np.array([0.05, -0.02, 0.01])
    Mt = np.diag([0.45, 0.42, 0.47]) + 0.01 * (np.ones((3, 3)) - np.eye(3))
    G = O.g_ansatz(np.array(th), np.array(M0), m, Mt)
    w = np.array([{0: 8 / 27, 1: 2 / 27, 2: 1 / 54, 3: 1 / 216}[int((c * c).sum())] for c in C])
    grad = w * (M0 + 3 * C @ m + 4.5 * np.einsum("ab,ia,ib->i", Mt - M0 * th * np.eye(3),
                                                   C, C) - 4.5 * th * np.trace(Mt - M0 * th * np.eye(3)))
    np.testing.assert_allclose(G, grad, atol=1e-14)


# ---------------------------------------------------------------------------
# Eqs. (f0mom)-(geq2mom) and (Pa): equilibrium moment constraints of the
# initial state, with P, H, E written in closed form from the inputs.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("M", [1, 2, 3, 8])
def test_equilibrium_moment_constraints(M):
    prm = _rand_params(M, seed=M)
    shape = (2, 3, 4)
    rng = np.random.Generator(np.random.PCG64(5))
    X = rng.uniform(0.1, 1.0, (M,) + shape)
    X /= X.sum(axis=0)
    u = rng.uniform(-0.1, 0.1, (3,) + shape)
    T = rng.uniform(0.3, 0.6, shape)
    P = rng.uniform(0.01, 0.05, shape)
    pops = O.init_populations(X, u, T, P, prm)
    C = O.C.astype(float)
    # closed forms
    mbar = np.einsum("a...,a->...", X, prm.molar_mass)
    Y = X * prm.molar_mass.reshape((M,) + (1,) * 3) / mbar
    rho = P * mbar / (prm.R_U * T)
    cv = np.einsum("a...,a->...", Y, prm.cv_molar * prm.R_U / prm.molar_mass)
    H = (cv + prm.R_U / mbar) * T
    usq = (u ** 2).sum(axis=0)
    rhoE = rho * (cv * T + usq / 2)
    for a in range(M):
        np.testing.assert_allclose(pops[a].sum(axis=0), Y[a] * rho, rtol=1e-13)
        np.testing.assert_allclose(np.einsum("i...,id->d...", pops[a], C), Y[a] * rho * u, atol=1e-15)
        Pa = Y[a] * rho * prm.R_U / prm.molar_mass[a] * T     # Eq. (eosIdeaGasComponent)
        sec = np.einsum("i...,ia,ib->ab...", pops[a], C, C)
        exp = Pa[None, None] * np.eye(3)[:, :, None, None, None] + Y[a] * rho * u[:, None] * u[None, :]
        np.testing.assert_allclose(sec, exp, atol=1e-15)       # Eq. (Pa)
    f, g = pops[M], pops[M + 1]
    np.testing.assert_allclose(f.sum(axis=0), rho, rtol=1e-13)
    Peq = P[None, None] * np.eye(3)[:, :, None, None, None] + rho * u[:, None] * u[None, :]
    np.testing.assert_allclose(np.einsum("i...,ia,ib->ab...", f, C, C), Peq, atol=1e-15)
    # Eq. (feq3mom) holds off the diagonal: Q_xxy = P u_y + rho u_x^2 u_y
    Qxxy = np.einsum("i...,i,i->...", f, C[:, 0] ** 2, C[:, 1])
    np.testing.assert_allclose(Qxxy, P * u[1] + rho * u[0] ** 2 * u[1], atol=1e-15)
    np.testing.assert_allclose(g.sum(axis=0), rhoE, rtol=1e-13)
    np.testing.assert_allclose(np.einsum("i...,id->d...", g, C), (H + usq / 2) * rho * u, atol=1e-14)
    Req = (H + usq / 2) * Peq + P * u[:, None] * u[None, :]
    np.testing.assert_allclose(np.einsum("i...,ia,ib->ab...", g, C, C), Req, atol=1e-14)
    # thermodynamic round trip, Eq. (temperature2) with T0 = 0
    st = O.node_state(O.moments(pops, prm), prm)
    np.testing.assert_allclose(st["T"], T, rtol=1e-13)
    np.testing.assert_allclose(st["P"], P, rtol=1e-13)
    np.testing.assert_allclose(st["X"], X, atol=1e-14)
    np.testing.assert_allclose(st["Cp"] - st["Cv"], st["R"], rtol=1e-13)   # Mayer


# ---------------------------------------------------------------------------
# Sec. 4.4, Eq. (soundTestConditions): printed mixture gas constants
# ---------------------------------------------------------------------------
def test_printed_mixture_gas_constants():
    masses = {"H2": 2.016, "Ar": 39.948, "CH4": 16.043, "C3H8": 44.097}
    mm = np.array(list(masses.values()))
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "sound_speed_mixture_R.txt"))
            if l.strip() and not l.startswith("#")]
    prm = O.Params(mm, np.full(4, 2.5), np.full((4, 4), 0.05) - 0.05 * np.eye(4),
                   omega_fixed=1.5, omega1_fixed=1.5)
    for name, R_printed, *X in rows:
        X = np.array([float(v) for v in X]).reshape(4, 1, 1, 1)
        pops = O.init_populations(X, np.zeros((3, 1, 1, 1)), np.full((1, 1, 1), 0.5),
                                  np.full((1, 1, 1), 0.02), prm)
        st = O.node_state(O.moments(pops, prm), prm)
        assert abs(st["R"].item() / float(R_printed) - 1.0) < 5e-5, name


# ---------------------------------------------------------------------------
# Collision invariants: Eqs. (densitya), (f0mom), (f1mom), (g0mom) and the
# momentum source A_i . X of Eq. (fwithcorrection); Sec. 3.5 coupling.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("coupling", ["strong", "weak"])
@pytest.mark.parametrize("M", [2, 3])
def test_collision_conservation(M, coupling):
    prm = _rand_params(M, coupling=coupling, seed=10 + M)
    pops = _rand_state(prm, (4, 5, 6), seed=M)
    post, aux = O.collide(pops, prm, return_aux=True)
    C = O.C.astype(float)
    d = post - pops
    tol = 1e-14 * np.abs(pops).max()
    for a in range(M):
        if coupling == "strong" and a == prm.slaved:
            continue
        np.testing.assert_allclose(d[a].sum(axis=0), 0.0, atol=tol)
    np.testing.assert_allclose(d[M].sum(axis=0), 0.0, atol=tol)
    np.testing.assert_allclose(np.einsum("i...,id->d...", d[M], C), aux["Xc"], atol=tol)
    np.testing.assert_allclose(d[M + 1].sum(axis=0), 0.0, atol=tol)
    # summation by parts: the correction source has zero grid sum
    np.testing.assert_allclose(aux["Xc"].sum(axis=(1, 2, 3)), 0.0, atol=tol)
    if coupling == "weak":
        tot = sum(np.einsum("i...,id->d...", d[a], C) for a in range(M))
        np.testing.assert_allclose(tot, 0.0, atol=tol)


@pytest.mark.parametrize("coupling", ["strong", "weak"])
@pytest.mark.parametrize("M", [2, 3, 5])
def test_stefan_maxwell_friction(M, coupling):
    """The momentum change of each species in the collision equals the
    Stefan-Maxwell friction sum_b (P X_a X_b / D_ab)(V_b - V_a) of Eq.
    (constit2) with theta_ab of Eq. (smDiffusionCoefficients2), and V solves
    Eq. (transform12) as printed."""
    prm = _rand_params(M, coupling=coupling, seed=30 + M)
    pops = _rand_state(prm, (3, 3, 4), seed=7 + M)
    post, aux = O.collide(pops, prm, return_aux=True)
    C = O.C.astype(float)
    V, X, rho_a = aux["V"], aux["X"], aux["rho_a"]
    Psp = aux["rho_sp"] * aux["R"] * aux["T"]       # pressure of the species subsystem
    for a in range(M):
        K = [Psp * X[a] * X[b] / prm.D[a, b] for b in range(M)]
        fric = sum(K[b][None] * (V[b] - V[a]) for b in range(M))
        # Eq. (transform12)
        lhs = rho_a[a][None] * V[a] - 0.5 * fric
        rhs = aux["j_a"][a] - rho_a[a][None] * aux["u_sp"]
        np.testing.assert_allclose(lhs, rhs, atol=1e-14 * np.abs(rhs).max())
        if coupling == "strong" and a == prm.slaved:
            continue
        dj = np.einsum("i...,id->d...", post[a] - pops[a], C)
        np.testing.assert_allclose(dj, fric, atol=1e-13 * np.abs(pops[a]).max())
    if coupling == "strong":
        flux = np.abs(np.stack([rho_a[a][None] * V[a] for a in range(M)])).max()
        scale = max(flux, np.abs(aux["j_a"]).max())
        np.testing.assert_allclose(sum(rho_a[a][None] * V[a] for a in range(M)), 0.0, atol=1e-14 * scale)


def test_binary_closed_form():
    """M = 2: J_1 = -J_2 = r_1 / (1 + (1/2)(P X_1 X_2 / D_12)(1/rho_1 + 1/rho_2))."""
    prm = _rand_params(2, seed=3)
    pops = _rand_state(prm, (2, 2, 3), seed=4)
    st = O.node_state(O.moments(pops, prm), prm)
    V = O.sm_momenta(st, prm)
    r1 = st["j_a"][0] - st["rho_a"][0] * st["u"]
    K = st["P"] * st["X"][0] * st["X"][1] / prm.D[0, 1]
    J1 = r1 / (1 + 0.5 * K * (1 / st["rho_a"][0] + 1 / st["rho_a"][1]))
    np.testing.assert_allclose(st["rho_a"][0] * V[0], J1, atol=1e-16)
    np.testing.assert_allclose(st["rho_a"][1] * V[1], -J1, atol=1e-16)


# ---------------------------------------------------------------------------
# Propagation and the lattice derivative
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(2, 2, 2), (3, 3, 3), (3, 4, 5)])
def test_stream_moves_each_population_along_its_link(shape):
    nz, ny, nx = shape
    for i in range(27):
        post = np.zeros((1, 27) + shape)
        z, y, x = 1 % nz, 2 % ny, 0
        post[0, i, z, y, x] = 1.0
        out = O.stream(post)
        c = O.C[i]
        dst = ((z + c[2]) % nz, (y + c[1]) % ny, (x + c[0]) % nx)
        assert out[0, i][dst] == 1.0 and out.sum() == 1.0


def test_isotropic_derivative_closed_forms():
    n = 16
    k = 2 * np.pi / n
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    f = np.sin(k * x)
    np.testing.assert_allclose(O.iso_derivative(f, 0), np.sin(k) * np.cos(k * x), atol=1e-14)
    np.testing.assert_allclose(O.iso_derivative(f, 1), 0.0, atol=1e-14)
    g = np.sin(k * x) * np.sin(k * y)
    exp = np.sin(k) * np.cos(k * x) * np.sin(k * y) * (2 + np.cos(k)) / 3
    np.testing.assert_allclose(O.iso_derivative(g, 0), exp, atol=1e-14)
    h = np.sin(k * z) * np.cos(k * y) * np.cos(k * x)
    exp = np.sin(k) * np.cos(k * z) * np.cos(k * y) * np.cos(k * x) * ((2 + np.cos(k)) / 3) ** 2
    np.testing.assert_allclose(O.iso_derivative(h, 2), exp, atol=1e-14)


# ---------------------------------------------------------------------------
# Sec. 3.3: transport closures
# ---------------------------------------------------------------------------
def test_transport_closed_forms():
    M = 3
    mm = np.array([20.0, 20.0, 20.0])
    mu0, lam0 = 0.003, 0.008
    prm = O.Params(mm, np.full(M, 2.5), np.full((M, M), 0.05), mu=np.full(M, mu0), lam=np.full(M, lam0))
    pops = _rand_state(prm, (2, 2, 2), seed=9, noise=0.0)
    st = O.node_state(O.moments(pops, prm), prm)
    P = st["P"]
    # identical species: phi_ab = 1, Wilke gives mu0; Mathur gives lam0
    np.testing.assert_allclose(st["omega"], 2 * P / (P + 2 * mu0), rtol=1e-14)
    np.testing.assert_allclose(st["omega1"], 2 * P * st["Cp"] / (P * st["Cp"] + 2 * lam0), rtol=1e-14)
    # Eq. (prandtl): Pr = omega1 (2 - omega) / (omega (2 - omega1)) = mu C_p / lambda
    w, w1 = st["omega"], st["omega1"]
    np.testing.assert_allclose(w1 * (2 - w) / (w * (2 - w1)), mu0 * st["Cp"] / lam0, rtol=1e-13)
    # Eq. (mu): mu = (1/omega - 1/2) P
    np.testing.assert_allclose((1 / w - 0.5) * P, mu0, rtol=1e-13)


def test_wilke_binary_textbook_value():
    """Wilke's rule for a binary mixture written out by hand for two species
    (phi_12, phi_21 from Eq. wilkePhi)."""
    m1, m2, mu1, mu2 = 2.0, 28.0, 0.9e-5, 1.8e-5
    x1 = 0.3
    p12 = (1 + (mu1 / mu2) ** 0.5 * (m2 / m1) ** 0.25) ** 2 / (8 * (1 + m1 / m2)) ** 0.5
    p21 = (1 + (mu2 / mu1) ** 0.5 * (m1 / m2) ** 0.25) ** 2 / (8 * (1 + m2 / m1)) ** 0.5
    mu_mix = x1 * mu1 / (x1 + (1 - x1) * p12) + (1 - x1) * mu2 / ((1 - x1) + x1 * p21)
    prm = O.Params(np.array([m1, m2]), np.array([2.5, 2.5]), np.array([[0, .05], [.05, 0]]),
                   mu=np.array([mu1, mu2]), lam=np.array([1.0, 1.0]))
    X = np.array([x1, 1 - x1]).reshape(2, 1, 1, 1)
    pops = O.init_populations(X, np.zeros((3, 1, 1, 1)), np.full((1, 1, 1), 0.5), np.full((1, 1, 1), 0.02), prm)
    st = O.node_state(O.moments(pops, prm), prm)
    P = st["P"].item()
    assert np.isclose((1 / st["omega"].item() - 0.5) * P, mu_mix, rtol=1e-12)


def test_mathur_binary_hand_value():
    """Eq. (conductivityMixture) with unequal species conductivities, worked
    by hand for X = (1/4, 3/4), lambda = (0.02, 0.004):
      sum X_a lambda_a = 0.005 + 0.003 = 0.008,
      sum X_a / lambda_a = 12.5 + 187.5 = 200,
      lambda = (0.008 + 1/200) / 2 = 0.0065,
    then Eq. (omega1).  The arithmetic mean alone (0.008), the harmonic one
    alone (0.005) or a missing 1/2 (0.013) all give another omega_1.  C_p is
    written out from Mayer's relation: (cv + 1) R_U / m_a per species, mixed
    by mass fraction."""
    m = np.array([4.0, 40.0])
    cv = np.array([1.5, 2.5])
    prm = O.Params(m, cv, np.array([[0, .05], [.05, 0]]), mu=np.array([1e-3, 1e-3]),
                   lam=np.array([0.02, 0.004]))
    X = np.array([0.25, 0.75]).reshape(2, 1, 1, 1)
    T, P = 0.3, 0.04
    pops = O.init_populations(X, np.zeros((3, 1, 1, 1)), np.full((1, 1, 1), T), np.full((1, 1, 1), P), prm)
    st = O.node_state(O.moments(pops, prm), prm)
    mbar = 0.25 * 4.0 + 0.75 * 40.0                       # 31
    Y = np.array([0.25 * 4.0, 0.75 * 40.0]) / mbar
    Cp = Y[0] * 2.5 / 4.0 + Y[1] * 3.5 / 40.0
    lam = 0.0065
    assert np.isclose(st["P"].item(), P, rtol=1e-13)
    assert np.isclose(st["Cp"].item(), Cp, rtol=1e-13)
    assert np.isclose(st["omega1"].item(), 2 * P * Cp / (P * Cp + 2 * lam), rtol=1e-12)
    # Eq. (lambda) read back: lambda = (1/omega_1 - 1/2) P C_p
    assert np.isclose((1 / st["omega1"].item() - 0.5) * P * Cp, lam, rtol=1e-12)


# ---------------------------------------------------------------------------
# Special case: identical species reduce to the single-component compressible
# model (Sec. 5, last paragraph): f and g do not depend on how the mass is split.
# ---------------------------------------------------------------------------
def test_identical_species_reduce_to_single_component():
    shape = (3, 4, 8)
    rng = np.random.Generator(np.random.PCG64(11))
    p2 = O.Params(np.array([16.0, 16.0]), np.array([2.5, 2.5]), np.array([[0, 0.03], [0.03, 0]]),
                  mu=np.array([0.002, 0.002]), lam=np.array([0.006, 0.006]))
    p1 = O.Params(np.array([16.0]), np.array([2.5]), np.array([[0.03]]),
                  mu=np.array([0.002]), lam=np.array([0.006]))
    X1 = rng.uniform(0.2, 0.8, shape)
    X = np.stack([X1, 1 - X1])
    u = rng.uniform(-0.05, 0.05, (3,) + shape)
    T = rng.uniform(0.45, 0.55, shape)
    P = rng.uniform(0.02, 0.03, shape)
    a = O.init_populations(X, u, T, P, p2)
    b = O.init_populations(np.ones((1,) + shape), u, T, P, p1)
    for _ in range(10):
        a = O.step(a, p2)
        b = O.step(b, p1)
    np.testing.assert_allclose(a[2:], b[1:], rtol=1e-12, atol=1e-15)


def test_patch_center_equals_full_grid():
    prm = _rand_params(3, seed=21)
    pops = _rand_state(prm, (7, 6, 9), seed=22)
    full = O.collide(pops, prm)
    for (z, y, x) in [(0, 0, 0), (3, 2, 5), (6, 5, 8)]:
        np.testing.assert_allclose(O.collide_patch_center(pops, z, y, x, prm), full[:, :, z, y, x],
                                   rtol=1e-14, atol=1e-16)
