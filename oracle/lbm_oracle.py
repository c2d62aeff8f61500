"""Plain FP64 NumPy oracle of one stream-and-collide step of the multicomponent
lattice Boltzmann model of Sawant, Dorschner & Karlin (arXiv 2004.11286).

TEST INFRASTRUCTURE ONLY: used by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``; never by the product path.  It is
deliberately slow and literal: every function follows one passage of the
paper, in the paper's order and notation, vectorised over grid nodes with
NumPy and nothing else (no blocking, fusion or reordering).

State layout (an interface convention shared with the C-ABI, not code):
``pops[L, i, z, y, x]`` with lattices ``L = 0..M-1`` the species populations
(the transformed ``k_ai`` of Sec. 2.5.2, renamed ``f_ai`` in Sec. 2.5.3),
``L = M`` the momentum lattice ``f`` and ``L = M+1`` the energy lattice ``g``.
Velocity index ``i = (cx+1) + 3(cy+1) + 9(cz+1)`` enumerates the D3Q27 set
of Eq. (d3q27vel); the rest velocity is ``i = 13`` and ``opp(i) = 26 - i``.
The populations are the post-streaming values at time t.  Lattice units
``dt = dx = 1`` throughout.

Readings taken where the paper is silent or singular (each also recorded in
the design notes):
  * the self-diffusivity D_aa (needed by the b = a terms of Eqs. tau and
    fStar) defaults to the geometric mean of row a's off-diagonal entries;
  * the isotropic derivative of Sec. 4.1 is the D3Q27 weighted central
    stencil d_a phi(x) = 3 sum_i w_i c_ia phi(x + c_i), periodic wrap;
  * all non-local inputs (grad Y_a, X_alpha) are moments of time t
    (synchronous evaluation);
  * strong coupling slaves species ``slaved`` (Eqs. rhoMATCH, uMATCH); its
    populations are still stored, streamed and relaxed with the slaved
    density and momentum; the sums of Eqs. rhoMATCH/uMATCH run over all i;
  * weak coupling: the species equilibria and the Stefan-Maxwell solve use
    the species' own density and velocity (Eqs. rhoSPEC, uSPEC);
  * the diffusion velocity of a species whose density is below 1e-14 of
    the mixture density is taken as zero (it only enters multiplied by
    rho_a);
  * at omega == omega_1 exactly, the (omega - omega_1)(g* - g) term of
    Eq. (g) is replaced by its limit (q_diff and q_corr carry a
    1/(omega - omega_1) factor);
  * walls (``walls_x``: the two faces normal to x, the closed tube of
    Sec. 4.2) reflect every lattice by halfway bounce-back: a population
    that would leave the domain returns to its node with the opposite
    velocity at the next time level.  The isotropic derivative reads the
    node outside a wall as the mirror image of the node inside it: even for
    the scalars, the y and z components and the G_alpha, odd for Phi_x (the
    wall-normal component of a momentum-like field).  The paper leaves both
    the derivative and the wall treatment of the three-dimensional model
    unstated.
  * the opposed-jets boundary set of Sec. 4.3 (``frame``, class Frame): a
    layer of nodes outside the x and y faces holds, after every collision,
    post-collision populations that then stream into the domain.  On the x
    faces, rows inside the nozzles hold the complete equilibrium of the
    inlet state (the incoming populations replaced by equilibria); the other
    rows are free-slip walls, the mirror image of the boundary node with the
    x velocity reflected (specular reflection halfway between the nodes).
    On the y faces (the outlets) the outside node is a copy of the boundary
    node (zero normal derivative).  An outside node beyond both faces takes
    the x-face rule of the boundary row it is next to.  The isotropic
    derivative reads an outside node as the value of its nearest boundary
    node, negated for Phi_x beyond a free-slip wall.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

Q = 27
# D3Q27 velocities, Eq. (d3q27vel): c_ia in {-1, 0, 1}.
C = np.array([[cx, cy, cz] for cz in (-1, 0, 1) for cy in (-1, 0, 1)
              for cx in (-1, 0, 1)], dtype=np.int64)
OPP = np.array([int(np.where((C == -C[i]).all(axis=1))[0][0]) for i in range(Q)])
_C2 = (C * C).sum(axis=1)           # |c_i|^2 in {0, 1, 2, 3}

# Weights of the isotropic gradient stencil (Sec. 4.1 reading): the standard
# D3Q27 lattice weights, by |c_i|^2.
_W_ISO = np.array([{0: 8.0 / 27, 1: 2.0 / 27, 2: 1.0 / 54, 3: 1.0 / 216}[int(s)]
                   for s in _C2])

RHO_EPS = 1e-14


@dataclass
class Params:
    """Problem statement of Secs. 2-3: species molar masses m_a, molar
    specific heats (constant, T0 = 0, Sec. 4.1), binary diffusivities D_ab
    (Eq. smDiffusionCoefficients2), species viscosities and conductivities
    (Wilke, Eq. viscosityMixture; Mathur, Eq. conductivityMixture) or fixed
    relaxation rates, and the coupling mode (Sec. 3.5)."""
    molar_mass: np.ndarray
    cv_molar: np.ndarray            # C-bar_{a,v} / R_U
    D: np.ndarray                   # (M, M), symmetric; diag <= 0 -> default
    mu: Optional[np.ndarray] = None
    lam: Optional[np.ndarray] = None
    omega_fixed: float = 0.0
    omega1_fixed: float = 0.0
    R_U: float = 1.0
    coupling: str = "strong"
    slaved: int = -1
    walls_x: bool = False           # bounce-back walls at x = -1/2 and x = nx - 1/2
    frame: Optional["Frame"] = None  # opposed-jets boundary set (Sec. 4.3)
    # temperature-dependent specific heats (Sec. 3.1): C-bar_{a,v}(T) / R_U =
    # sum_k cv_poly[a, k] T^k; None: the constants cv_molar (T0 = 0 either way)
    cv_poly: Optional[np.ndarray] = None
    M: int = field(init=False)

    def __post_init__(self):
        self.molar_mass = np.asarray(self.molar_mass, dtype=np.float64)
        self.cv_molar = np.asarray(self.cv_molar, dtype=np.float64)
        self.M = int(self.molar_mass.shape[0])
        D = np.array(self.D, dtype=np.float64).reshape(self.M, self.M)
        assert np.allclose(D, D.T), "D_ab must be symmetric"
        for a in range(self.M):
            if D[a, a] <= 0.0:
                off = [D[a, b] for b in range(self.M) if b != a]
                if not off:
                    raise ValueError("M = 1 needs an explicit D_11 > 0")
                D[a, a] = float(np.exp(np.mean(np.log(off))))
        self.D = D
        if self.mu is not None:
            self.mu = np.asarray(self.mu, dtype=np.float64)
        if self.lam is not None:
            self.lam = np.asarray(self.lam, dtype=np.float64)
        if self.slaved < 0:
            self.slaved = self.M - 1
        assert self.coupling in ("strong", "weak")
        assert not (self.walls_x and self.frame is not None), "walls_x and frame exclude each other"
        if self.cv_poly is not None:
            self.cv_poly = np.asarray(self.cv_poly, dtype=np.float64).reshape(self.M, -1)

    @property
    def S(self) -> int:
        return self.M + 2

    @property
    def R_a(self) -> np.ndarray:
        """Species gas constants, Eq. (Ra)."""
        return self.R_U / self.molar_mass

    @property
    def Cv_a(self) -> np.ndarray:
        """Mass-based C_{a,v} = C-bar_{a,v} / m_a (Sec. 3.1)."""
        return self.cv_molar * self.R_U / self.molar_mass

    @property
    def Cp_a(self) -> np.ndarray:
        """Mayer's relation in the mass basis, C_{a,p} - C_{a,v} = R_a (Sec. 3.1)."""
        return self.Cv_a + self.R_a

    def _coef(self) -> np.ndarray:
        """(M, K) coefficients of C-bar_{a,v}(T) / R_U in powers of T."""
        return self.cv_poly if self.cv_poly is not None else self.cv_molar[:, None]

    def cv_a_of(self, T) -> np.ndarray:
        """C_{a,v}(T) = C-bar_{a,v}(T) / m_a per species, shape (M,) + T.shape."""
        T = np.asarray(T, dtype=np.float64)
        c = self._coef()
        out = np.zeros((self.M,) + T.shape)
        for k in range(c.shape[1]):
            out = out + (c[:, k] * self.R_U / self.molar_mass).reshape((self.M,) + (1,) * T.ndim) * T[None] ** k
        return out

    def U_a_of(self, T) -> np.ndarray:
        """Eq. (specUa) with T0 = 0: U_a(T) = int_0^T C_{a,v}(T') dT', the
        polynomial's integral term by term."""
        T = np.asarray(T, dtype=np.float64)
        c = self._coef()
        out = np.zeros((self.M,) + T.shape)
        for k in range(c.shape[1]):
            out = out + (c[:, k] * self.R_U / self.molar_mass / (k + 1)).reshape((self.M,) + (1,) * T.ndim) \
                * T[None] ** (k + 1)
        return out

    def H_a_of(self, T) -> np.ndarray:
        """Eq. (specHa) with T0 = 0: H_a(T) = int_0^T C_{a,p} dT' = U_a(T) + R_a T
        (Mayer's relation in the mass basis)."""
        T = np.asarray(T, dtype=np.float64)
        return self.U_a_of(T) + self.R_a.reshape((self.M,) + (1,) * T.ndim) * T[None]


# ----------------------------------------------------------------------------
# Product-form and energy-lattice ansatz (Secs. 2.4 and 3.4.1)
# ----------------------------------------------------------------------------

def _psi_1d(c: int, xi, zeta):
    """The triplet Psi_0, Psi_{+1}, Psi_{-1} of Sec. 2.4."""
    if c == 0:
        return 1.0 - (xi * xi + zeta)
    return (c * xi + (xi * xi + zeta)) / 2.0


def psi_product(xi, zeta):
    """Eq. (prod): Psi_i(xi, zeta) = prod_alpha Psi_{c_ia}(xi_alpha, zeta).
    ``xi`` has shape (3, ...), ``zeta`` shape (...). Returns (27, ...)."""
    xi = np.asarray(xi, dtype=np.float64)
    zeta = np.asarray(zeta, dtype=np.float64)
    out = np.empty((Q,) + zeta.shape)
    for i in range(Q):
        out[i] = (_psi_1d(C[i, 0], xi[0], zeta) * _psi_1d(C[i, 1], xi[1], zeta)
                  * _psi_1d(C[i, 2], xi[2], zeta))
    return out


def _w_1d(c: int, theta):
    """Eq. (w0): w_0 = 1 - theta, w_{+-1} = theta / 2."""
    return 1.0 - theta if c == 0 else theta / 2.0


def g_ansatz(theta, M0, m, Mt):
    """Eqs. (gansatz), (grad), (weights), (RcorrectionPrime), (Bi):
    G_i = h_i + B_i . Z with product weights w_i(theta).
    Shapes: theta, M0 (...); m (3, ...); Mt (3, 3, ...). Returns (27, ...)."""
    theta = np.asarray(theta, dtype=np.float64)
    M0 = np.asarray(M0, dtype=np.float64)
    out = np.empty((Q,) + theta.shape)
    Z = [(1.0 - 3.0 * theta) / (2.0 * theta) * (Mt[a, a] - theta * M0) for a in range(3)]
    for i in range(Q):
        c = C[i]
        w = _w_1d(c[0], theta) * _w_1d(c[1], theta) * _w_1d(c[2], theta)
        mc = m[0] * c[0] + m[1] * c[1] + m[2] * c[2]
        second = np.zeros_like(theta)
        for a in range(3):
            for b in range(3):
                delta = 1.0 if a == b else 0.0
                second = second + (Mt[a, b] - M0 * theta * delta) * (c[a] * c[b] - theta * delta)
        h = w * (M0 + mc / theta + second / (2.0 * theta * theta))
        if _C2[i] == 0:
            B = (1.0, 1.0, 1.0)
        elif _C2[i] == 1:
            B = tuple(-0.5 * abs(int(c[a])) for a in range(3))
        else:
            B = (0.0, 0.0, 0.0)
        out[i] = h + B[0] * Z[0] + B[1] * Z[1] + B[2] * Z[2]
    return out


# ----------------------------------------------------------------------------
# Lattice operators
# ----------------------------------------------------------------------------

XREF = np.array([int(np.where((C == C[i] * np.array([-1, 1, 1])).all(axis=1))[0][0]) for i in range(Q)])


@dataclass
class Frame:
    """Boundary set of the opposed jets (Sec. 4.3; the readings are in the
    module docstring).  y0, y1: the interior rows [y0, y1) of both x faces that
    are nozzles; inlet: the complete populations (S, 27) entering through
    the nozzle at x = -1 (inlet[0]) and at x = nx (inlet[1]).  x_faces /
    y_faces False leave that pair of faces periodic."""
    y0: int
    y1: int
    inlet: tuple = ()
    x_faces: bool = True
    y_faces: bool = True


def _frame_rows(ny: int, fr: Frame):
    """For each row yp of the padded grid (yp = y + 1), the interior row it
    takes its values from: the nearest one beyond outlets, the wrapped one
    beyond periodic y faces."""
    yp = np.arange(ny + 2) - 1
    return np.clip(yp, 0, ny - 1) if fr.y_faces else yp % ny


def _frame_pad_pops(post, fr: Frame):
    """Post-collision populations (S, 27, nz, ny, nx) with one layer of outside
    nodes on the x and y faces, (S, 27, nz, ny + 2, nx + 2)."""
    S, _, nz, ny, nx = post.shape
    pad = np.empty((S, Q, nz, ny + 2, nx + 2))
    pad[..., 1:-1, 1:-1] = post
    if fr.y_faces:                              # outlets: copies of the boundary rows
        pad[..., 0, 1:-1] = post[..., 0, :]
        pad[..., -1, 1:-1] = post[..., -1, :]
    else:
        pad[..., 0, 1:-1] = post[..., -1, :]
        pad[..., -1, 1:-1] = post[..., 0, :]
    if not fr.x_faces:
        pad[..., 0] = pad[..., nx]
        pad[..., -1] = pad[..., 1]
        return pad
    rows = _frame_rows(ny, fr)
    for yp in range(ny + 2):
        yc = int(rows[yp])
        for side, xo, xb in ((0, 0, 0), (1, nx + 1, nx - 1)):
            if fr.y0 <= yc < fr.y1:             # nozzle: the inlet equilibrium
                pad[:, :, :, yp, xo] = np.asarray(fr.inlet[side])[:, :, None]
            else:                               # free-slip wall: x velocity reflected
                pad[:, :, :, yp, xo] = post[:, XREF][:, :, :, yc, xb]
    return pad


def _frame_pad_field(phi, fr: Frame, odd_x: bool = False):
    """A field (..., nz, ny, nx) with one layer of outside nodes: the nearest
    boundary node's value (wrapped on periodic faces), negated beyond a
    free-slip wall for a field odd in x."""
    ny, nx = phi.shape[-2], phi.shape[-1]
    pad = np.empty(phi.shape[:-2] + (ny + 2, nx + 2))
    rows = _frame_rows(ny, fr)
    inner = phi[..., rows, :]                   # (..., ny + 2, nx)
    pad[..., 1:-1] = inner
    if not fr.x_faces:
        pad[..., 0] = inner[..., -1]
        pad[..., -1] = inner[..., 0]
        return pad
    nozzle = (rows >= fr.y0) & (rows < fr.y1)
    sgn = np.where(nozzle, 1.0, -1.0) if odd_x else np.ones(ny + 2)
    pad[..., 0] = sgn * inner[..., 0]
    pad[..., -1] = sgn * inner[..., -1]
    return pad


def stream_frame(post, fr: Frame):
    """Propagation with the opposed-jets boundary set: every population moves
    from x - c_i to x, those from outside the domain taken from the outside
    layer of _frame_pad_pops."""
    pad = _frame_pad_pops(post, fr)
    out = np.empty_like(post)
    for i in range(Q):
        sh = np.roll(pad[:, i], shift=(int(C[i, 2]), int(C[i, 1]), int(C[i, 0])), axis=(-3, -2, -1))
        out[:, i] = sh[..., 1:-1, 1:-1]
    return out


def _shift(phi, c, walls_x: bool = False, odd_x: bool = False):
    """phi(x + c); phi has shape (..., nz, ny, nx).  Periodic in every
    direction, or, with walls_x, mirrored across the two x walls: the node
    outside a wall takes the value of its mirror image inside, negated for a
    field that is odd in x."""
    out = np.roll(phi, shift=(-int(c[2]), -int(c[1])), axis=(-3, -2))
    if not walls_x or int(c[0]) == 0:
        return np.roll(out, shift=-int(c[0]), axis=-1)
    nx = phi.shape[-1]
    src = np.arange(nx) + int(c[0])
    outside = (src < 0) | (src >= nx)
    src = np.clip(src, 0, nx - 1)      # mirror image of x = -1 is 0, of x = nx is nx - 1
    out = out[..., src]
    if odd_x:
        out = np.where(outside, -out, out)
    return out


def iso_derivative(phi, alpha: int, walls_x: bool = False, odd_x: bool = False, frame: Optional[Frame] = None):
    """Second-order isotropic lattice derivative of Sec. 4.1 (reading):
    d_alpha phi(x) = 3 sum_i w_i c_{i alpha} phi(x + c_i)."""
    if frame is not None:
        pad = _frame_pad_field(phi, frame, odd_x)
        acc = np.zeros_like(pad, dtype=np.float64)
        for i in range(Q):
            if C[i, alpha] != 0:
                acc = acc + _W_ISO[i] * C[i, alpha] * np.roll(pad, shift=(-int(C[i, 2]), -int(C[i, 1]), -int(C[i, 0])),
                                                              axis=(-3, -2, -1))
        return 3.0 * acc[..., 1:-1, 1:-1]
    acc = np.zeros_like(phi, dtype=np.float64)
    for i in range(Q):
        if C[i, alpha] != 0:
            acc = acc + _W_ISO[i] * C[i, alpha] * _shift(phi, C[i], walls_x, odd_x)
    return 3.0 * acc


def stream(post, walls_x: bool = False):
    """Propagation along the links: the value at x in direction i moves to
    x + c_i (left-hand sides of Eqs. SMlbm, f, g). ``post`` (S, 27, nz, ny, nx).
    With walls_x, the value that would cross an x wall stays at its node and
    arrives there with the opposite velocity (halfway bounce-back)."""
    out = np.empty_like(post)
    for i in range(Q):
        out[:, i] = np.roll(post[:, i], shift=(int(C[i, 2]), int(C[i, 1]), int(C[i, 0])),
                            axis=(-3, -2, -1))
    if walls_x:
        for i in range(Q):
            if C[i, 0] > 0:        # arrives at x = 0 from outside: x's own value in -c_i
                out[:, i, :, :, 0] = post[:, OPP[i], :, :, 0]
            elif C[i, 0] < 0:      # arrives at x = nx - 1 from outside
                out[:, i, :, :, -1] = post[:, OPP[i], :, :, -1]
    return out


# ----------------------------------------------------------------------------
# Moments, coupling, thermodynamics and transport
# ----------------------------------------------------------------------------

def moments(pops, prm: Params):
    """Raw moments: species density and momentum (Eqs. densitya, auxua),
    mixture density, momentum and pressure tensor of the momentum lattice
    (Eqs. f0momDensity, f1momMomentum, boldP), total energy and energy flux
    of the energy lattice (Eqs. g0momTotalEnergy, q)."""
    M = prm.M
    Cf = C.astype(np.float64)
    k, f, g = pops[:M], pops[M], pops[M + 1]
    out = {}
    out["rho_a"] = k.sum(axis=1)
    out["j_a"] = np.einsum("ai...,id->ad...", k, Cf)
    out["rho"] = f.sum(axis=0)
    out["j"] = np.einsum("i...,id->d...", f, Cf)
    out["Pi"] = np.einsum("i...,id,ie->de...", f, Cf, Cf)
    out["rhoE"] = g.sum(axis=0)
    out["q"] = np.einsum("i...,id->d...", g, Cf)
    return out


def node_state(mom, prm: Params):
    """Per-node closure: coupling (Sec. 3.5), composition and equation of state
    (Sec. 2.1), caloric relations with constant specific heats and T0 = 0
    (Sec. 3.1, Eq. temperature2, Sec. 4.1), transport (Wilke, Mathur) and the
    relaxation rates (Eqs. omega, omega1)."""
    M = prm.M
    st = dict(mom)
    rho_a = mom["rho_a"].copy()
    j_a = mom["j_a"].copy()
    rho, j = mom["rho"], mom["j"]
    if prm.coupling == "strong":
        # Eqs. (rhoMATCH), (uMATCH): the slaved species takes the deficit.
        s = prm.slaved
        others = [a for a in range(M) if a != s]
        rho_a[s] = rho - rho_a[others].sum(axis=0)
        j_a[s] = j - j_a[others].sum(axis=0)
        rho_sp = rho
        u_sp = j / rho
    else:
        # Eqs. (rhoSPEC), (uSPEC): the species subsystem's own density/velocity.
        rho_sp = rho_a.sum(axis=0)
        u_sp = j_a.sum(axis=0) / rho_sp
    u = j / rho
    Y = rho_a / rho_sp                                          # Eq. (mixtureDensity)
    inv_m = np.einsum("a...,a->...", Y, 1.0 / prm.molar_mass)   # Eq. (meanMolecularWeight)
    m = 1.0 / inv_m
    X = Y * (m[None] / prm.molar_mass.reshape((M,) + (1,) * m.ndim))  # Eq. (moleFractionDefinition)
    R = prm.R_U / m                                             # Eq. (defineSpecificGasContant)
    usq = (u * u).sum(axis=0)
    if prm.cv_poly is None:
        Cv = np.einsum("a...,a->...", Y, prm.Cv_a)             # Eq. (Cvmix)
        Cp = np.einsum("a...,a->...", Y, prm.Cp_a)
        T = (mom["rhoE"] / rho - 0.5 * usq) / Cv                # Eq. (temperature2), T0 = 0
    else:
        T = temperature_from_energy(Y, mom["rhoE"] / rho - 0.5 * usq, prm)   # Eq. (temperature)
        Cv = np.einsum("a...,a...->...", Y, prm.cv_a_of(T))
        Cp = Cv + R
    P = rho * R * T                                             # Eq. (eosIdealGas)
    st.update(rho_a=rho_a, j_a=j_a, rho_sp=rho_sp, u_sp=u_sp, u=u, Y=Y, m=m, X=X,
              R=R, Cv=Cv, Cp=Cp, T=T, P=P, usq=usq)

    if prm.omega_fixed > 0.0:
        omega = np.full_like(rho, prm.omega_fixed)
    else:
        # Wilke mixture viscosity, Eqs. (viscosityMixture), (wilkePhi).
        mu_a, ma = prm.mu, prm.molar_mass
        phi = np.empty((M, M))
        for a in range(M):
            for b in range(M):
                phi[a, b] = ((1.0 + np.sqrt((mu_a[a] / mu_a[b]) * np.sqrt(ma[b] / ma[a]))) ** 2
                             / (np.sqrt(8.0) * np.sqrt(1.0 + ma[a] / ma[b])))
        mu_mix = np.zeros_like(rho)
        for a in range(M):
            den = np.zeros_like(rho)
            for b in range(M):
                den = den + phi[a, b] * X[b]
            mu_mix = mu_mix + mu_a[a] * X[a] / den
        omega = 2.0 * P / (P + 2.0 * mu_mix)                    # Eq. (omega), dt = 1
    if prm.omega1_fixed > 0.0:
        omega1 = np.full_like(rho, prm.omega1_fixed)
    else:
        # Mathur mixture conductivity, Eq. (conductivityMixture).
        lam_a = prm.lam
        s1 = np.einsum("a...,a->...", X, lam_a)
        s2 = np.einsum("a...,a->...", X, 1.0 / lam_a)
        lam_mix = 0.5 * (s1 + 1.0 / s2)
        omega1 = 2.0 * P * Cp / (P * Cp + 2.0 * lam_mix)        # Eq. (omega1), dt = 1
    st.update(omega=omega, omega1=omega1)
    return st


def temperature_from_energy(Y, e, prm: Params, tol: float = 1e-15, maxit: int = 60):
    """Eq. (temperature) with T0 = 0: the T that solves
    sum_a Y_a U_a(T) = e  (e = E - u^2/2), by Newton's method from the
    estimate of the specific heats at T = 0.  U is increasing (C_v > 0), so
    the iteration converges; it stops when the correction is below tol of T."""
    e = np.asarray(e, dtype=np.float64)
    cv0 = np.einsum("a...,a...->...", Y, prm.cv_a_of(np.zeros_like(e)))
    T = e / cv0
    for _ in range(maxit):
        U = np.einsum("a...,a...->...", Y, prm.U_a_of(T))
        Cv = np.einsum("a...,a...->...", Y, prm.cv_a_of(T))
        dT = (U - e) / Cv
        T = T - dT
        if np.all(np.abs(dT) <= tol * np.abs(T)):
            break
    return T


def inv_tau_ab(st, prm: Params):
    """Eq. (tauab): 1/tau_ab = (R_U T / D_ab) (m / (m_a m_b)), all a, b."""
    M = prm.M
    out = np.empty((M, M) + st["T"].shape)
    for a in range(M):
        for b in range(M):
            out[a, b] = (prm.R_U * st["T"] / prm.D[a, b]) * (
                st["m"] / (prm.molar_mass[a] * prm.molar_mass[b]))
    return out


def sm_momenta(st, prm: Params, itab=None):
    """Species velocities u_a(f) from Eq. (transform1):
    rho_a u_a(f) (1 + 1/(2 tau_a)) - (1/2) Y_a sum_b (1/tau_ab) rho_b u_b(f)
        = rho_a u_a(k),
    one M x M linear system per node, three right-hand sides (the components).
    Returns the diffusion velocities V_a = u_a(f) - u (Sec. 2.5.3)."""
    M = prm.M
    if itab is None:
        itab = inv_tau_ab(st, prm)
    Y = st["Y"]
    inv_tau_a = np.einsum("ab...,b...->a...", itab, Y)          # Eq. (tau)
    shape = st["T"].shape
    n = int(np.prod(shape)) if shape else 1
    A = np.zeros((n, M, M))
    for a in range(M):
        for b in range(M):
            val = -0.5 * Y[a] * itab[a, b]
            if a == b:
                val = val + 1.0 + 0.5 * inv_tau_a[a]
            A[:, a, b] = val.reshape(n)
    rhs = st["j_a"].reshape(M, 3, n).transpose(2, 0, 1)         # (n, M, 3)
    p = np.linalg.solve(A, rhs)                                 # rho_a u_a(f)
    p = p.transpose(1, 2, 0).reshape((M, 3) + shape)
    rho_a = st["rho_a"]
    ok = rho_a > RHO_EPS * st["rho_sp"]
    safe = np.where(ok, rho_a, 1.0)
    V = np.where(ok[:, None], p / safe[:, None] - st["u_sp"][None], 0.0)
    return V


# ----------------------------------------------------------------------------
# Collision
# ----------------------------------------------------------------------------

def collide(pops, prm: Params, return_aux: bool = False):
    """Post-collision populations at every node (before propagation) for the
    species (Eqs. SMlbm, fstar1, transform12), the momentum lattice with the
    D3Q27 correction (Eqs. feq, fwithcorrection, Xalpha, Ai) and the energy
    lattice (Eqs. g, gieq, gistar, gstareq1mom, interdiffusion, corrFourier)."""
    M = prm.M
    mom = moments(pops, prm)
    st = node_state(mom, prm)
    rho, j, u, T, P, R = st["rho"], st["j"], st["u"], st["T"], st["P"], st["R"]
    omega, omega1 = st["omega"], st["omega1"]

    # --- non-local fields (Sec. 4.1 derivatives of time-t moments) ---------
    wx, fr = prm.walls_x, prm.frame
    Phi = [j[a] * (1.0 - 3.0 * R * T) - rho * u[a] ** 3 for a in range(3)]
    c_om = 1.0 / omega - 0.5
    Gs = [c_om * iso_derivative(Phi[a], a, wx, odd_x=(a == 0), frame=fr) for a in range(3)]
    Xc = np.stack([-iso_derivative(Gs[a], a, wx, frame=fr) for a in range(3)])  # Eq. (Xalpha)
    gradY = np.stack([np.stack([iso_derivative(st["Y"][a], b, wx, frame=fr) for b in range(3)])
                      for a in range(M)])                              # (M, 3, ...)

    # --- species, Eqs. (tauab), (tau), beta_a, (SMlbm), (fstar1) ------------
    itab = inv_tau_ab(st, prm)
    V = sm_momenta(st, prm, itab)
    inv_tau_a = np.einsum("ab...,b...->a...", itab, st["Y"])
    beta = 1.0 / (2.0 / inv_tau_a + 1.0)                       # dt / (2 tau_a + dt)
    feq_s = np.stack([st["rho_a"][a] * psi_product(st["u_sp"], prm.R_a[a] * T)
                      for a in range(M)])
    fstar_s = np.stack([st["rho_a"][a] * psi_product(st["u_sp"] + V[a], prm.R_a[a] * T)
                        for a in range(M)])
    diff = feq_s - fstar_s
    post = np.empty_like(pops)
    for a in range(M):
        F = np.zeros_like(diff[0])
        for b in range(M):
            F = F + itab[a, b] * diff[b]
        F = st["Y"][a] * F
        k = pops[a]
        post[a] = k + 2.0 * beta[a] * (feq_s[a] - k) + (beta[a] - 1.0) * F

    # --- momentum lattice, Eqs. (feq), (fwithcorrection), (Ai) ---------------
    f = pops[M]
    feq = rho * psi_product(u, R * T)
    corr = np.zeros_like(f)
    for i in range(Q):
        if _C2[i] == 1:
            corr[i] = 0.5 * (C[i, 0] * Xc[0] + C[i, 1] * Xc[1] + C[i, 2] * Xc[2])
    post[M] = f + omega * (feq - f) + corr

    # --- energy lattice, Eqs. (g), (geq1mom), (geq2mom), (gstareq1mom) -------
    g = pops[M + 1]
    theta = R * T
    if prm.cv_poly is None:
        H_a = np.stack([prm.Cp_a[a] * T for a in range(M)])   # Eq. (specHa), constant heats, T0 = 0
        H = st["Cp"] * T                                       # Eq. (specH)
    else:
        H_a = prm.H_a_of(T)                                    # Eq. (specHa), T0 = 0
        H = np.einsum("a...,a...->...", st["Y"], H_a)         # Eq. (specH)
    eye = np.eye(3)
    Peq = np.empty((3, 3) + rho.shape)
    for a in range(3):
        for b in range(3):
            Peq[a, b] = P * eye[a, b] + rho * u[a] * u[b]       # Eq. (feq2mom)
    hk = H + 0.5 * st["usq"]
    qeq = hk[None] * j                                          # Eq. (geq1mom)
    Req = np.empty_like(Peq)
    for a in range(3):
        for b in range(3):
            Req[a, b] = hk * Peq[a, b] + P * u[a] * u[b]        # Eq. (geq2mom)
    geq = g_ansatz(theta, st["rhoE"], qeq, Req)                # Eq. (gieq)

    Pi = st["Pi"]
    qb = np.stack([st["q"][a] - sum(u[b] * (Pi[b, a] - Peq[b, a]) for b in range(3))
                   for a in range(3)])
    sHYV = sum(H_a[a][None] * st["Y"][a][None] * V[a] for a in range(M))
    sHgY = sum(H_a[a][None] * gradY[a] for a in range(M))
    dw = omega - omega1
    nonzero = dw != 0.0
    dw_safe = np.where(nonzero, dw, 1.0)
    qdiff = (omega1 / dw_safe)[None] * rho[None] * sHYV        # Eq. (interdiffusion)
    qcorr = (0.5 * (omega1 - 2.0) / (-dw_safe) * P)[None] * sHgY  # Eq. (corrFourier)
    qstar = qb + qdiff + qcorr                                  # Eq. (gstareq1mom)
    gstar = g_ansatz(theta, st["rhoE"], qstar, Req)            # Eq. (gistar)
    relax_star = dw * (gstar - g)
    if not nonzero.all():
        # Limit omega -> omega_1: G is affine in m, so (omega - omega_1)(g* - g)
        # -> w_i(theta) c_i . [omega_1 rho sum H_a Y_a V_a
        #                      + (1/2)(2 - omega_1) P sum H_a grad Y_a] / theta.
        flux = omega1[None] * rho[None] * sHYV + (0.5 * (2.0 - omega1) * P)[None] * sHgY
        lim = np.empty_like(g)
        for i in range(Q):
            c = C[i]
            w = _w_1d(c[0], theta) * _w_1d(c[1], theta) * _w_1d(c[2], theta)
            lim[i] = w * (c[0] * flux[0] + c[1] * flux[1] + c[2] * flux[2]) / theta
        relax_star = np.where(nonzero[None], relax_star, lim)
    post[M + 1] = g + omega1 * (geq - g) + relax_star

    if return_aux:
        aux = dict(st)
        aux.update(V=V, Xc=Xc, gradY=gradY, beta=beta, itab=itab, feq_s=feq_s,
                   fstar_s=fstar_s, feq=feq, geq=geq, gstar=gstar, qstar=qstar, Peq=Peq,
                   qeq=qeq, Req=Req, Phi=np.stack(Phi), G=np.stack(Gs))
        return post, aux
    return post


def step(pops, prm: Params):
    """One time step: collide at every node, then stream (Eqs. SMlbm, fwithcorrection, g)."""
    if prm.frame is not None:
        return stream_frame(collide(pops, prm), prm.frame)
    return stream(collide(pops, prm), prm.walls_x)


def run(pops, prm: Params, nsteps: int):
    for _ in range(nsteps):
        pops = step(pops, prm)
    return pops


# ----------------------------------------------------------------------------
# Initialisation and outputs
# ----------------------------------------------------------------------------

def init_populations(X, u, T, P, prm: Params):
    """Equilibrium initial state from mole fractions, velocity, temperature
    and pressure.  Species: f^eq_a = rho_a Psi(u, R_a T) (Eq. 27eq), which by
    Eq. (fixed) is also the equilibrium of the transformed populations.
    Momentum lattice: rho Psi(u, RT) (Eq. feq).  Energy lattice: g^eq of
    Eq. (gieq).  X (M, ...), u (3, ...), T and P (...)."""
    M = prm.M
    X = np.asarray(X, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    P = np.asarray(P, dtype=np.float64)
    mm = prm.molar_mass.reshape((M,) + (1,) * T.ndim)
    m = (X * mm).sum(axis=0)                       # 1/m = sum Y_a/m_a  <=>  m = sum X_a m_a
    Y = X * mm / m[None]
    R = prm.R_U / m
    rho = P / (R * T)
    rho_a = Y * rho[None]
    j = rho[None] * u
    usq = (u * u).sum(axis=0)
    if prm.cv_poly is None:
        Cv = np.einsum("a...,a->...", Y, prm.Cv_a)
        Cp = np.einsum("a...,a->...", Y, prm.Cp_a)
        rhoE = rho * (Cv * T + 0.5 * usq)
        H = Cp * T
    else:
        rhoE = rho * (np.einsum("a...,a...->...", Y, prm.U_a_of(T)) + 0.5 * usq)   # rho (U + u^2/2), Eq. (Umix)
        H = np.einsum("a...,a...->...", Y, prm.H_a_of(T))                          # Eq. (specH)
    pops = np.empty((M + 2, Q) + T.shape)
    for a in range(M):
        pops[a] = rho_a[a] * psi_product(u, prm.R_a[a] * T)
    pops[M] = rho * psi_product(u, R * T)
    hk = H + 0.5 * usq
    eye = np.eye(3)
    Peq = np.empty((3, 3) + T.shape)
    Req = np.empty((3, 3) + T.shape)
    for a in range(3):
        for b in range(3):
            Peq[a, b] = P * eye[a, b] + rho * u[a] * u[b]
    for a in range(3):
        for b in range(3):
            Req[a, b] = hk * Peq[a, b] + P * u[a] * u[b]
    pops[M + 1] = g_ansatz(R * T, rhoE, hk[None] * j, Req)
    return pops


def macroscopic(pops, prm: Params):
    """Observable fields of the state: rho, u, T, P, X_a, Y_a and the diffusion
    velocities V_a (the species velocity is u + V_a, Sec. 2.5.3)."""
    st = node_state(moments(pops, prm), prm)
    V = sm_momenta(st, prm)
    return dict(rho=st["rho"], u=st["u"], T=st["T"], P=st["P"], X=st["X"], Y=st["Y"], V=V,
                omega=st["omega"], omega1=st["omega1"])


def collide_patch_center(pops, z: int, y: int, x: int, prm: Params, radius: int = 2):
    """Post-collision populations of the single node (z, y, x) of a periodic
    grid, computed by ``collide`` on the (2r+1)^3 periodic neighbourhood.  The
    non-local terms reach two nodes away (X_alpha differentiates twice), so
    r = 2 reproduces the full-grid result exactly at the centre."""
    nz, ny, nx = pops.shape[-3:]
    iz = (np.arange(z - radius, z + radius + 1)) % nz
    iy = (np.arange(y - radius, y + radius + 1)) % ny
    ix = (np.arange(x - radius, x + radius + 1)) % nx
    patch = pops[:, :, iz][:, :, :, iy][:, :, :, :, ix]
    post = collide(np.ascontiguousarray(patch), prm)
    return post[:, :, radius, radius, radius]


def conserved_sums(pops, prm: Params):
    """Grid sums of every stored lattice's density, the mixture momentum and
    the total energy: [sum rho_a (a = 1..M), sum rho, sum j (3), sum rhoE]."""
    mom = moments(pops, prm)
    out = [mom["rho_a"][a].sum() for a in range(prm.M)]
    out.append(mom["rho"].sum())
    out.extend(mom["j"][d].sum() for d in range(3))
    out.append(mom["rhoE"].sum())
    return np.array(out)
