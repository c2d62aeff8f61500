"""Seeded synthetic workloads shaped like the paper's benchmarks (Sec. 4).

This module only draws and lays out INPUTS: species constants, transport
inputs and the initial macroscopic fields (mole fractions, velocity,
temperature, pressure) as float64 NumPy arrays.  It contains none of the
method's arithmetic (no equilibria, no moments, no collision), so both the
CUDA path and the CPU oracle can be fed from it.

Recipes (stand-ins for the paper's experiments; lattice units, R_U = 1):
  * ``ternary_tube``   -- periodic analogue of the Loschmidt tube of Sec. 4.2
    (64x4x4, m = 2, 40, 16, D12 = D13 = 0.05, D23 = 0.01, left/right mole
    fractions (0.5, 0.5, 0) / (0.5, 0, 0.5) joined by tanh steps).  The tanh
    scale is 8 cells rather than 2: with a 2-cell step the trace species in
    the tails diffuse at V ~ 2 D / width (Stefan-Maxwell, V = -D grad ln X),
    faster than the heavy species' lattice thermal speed sqrt(R_a T), and the
    product-form quasi-equilibrium turns negative and diverges (FP64 oracle,
    any T in 0.2..1.5).
  * ``acoustic_pulse`` -- binary sound-speed test after Sec. 4.4 (128^3,
    m = 4, 40, uniform X_1, Gaussian pressure pulse of amplitude 1e-3 and
    standard deviation 6 cells at the centre).
  * ``shear_layer``    -- periodic double shear layer after Sec. 4.5 (256^3,
    m = 2, 28, tanh velocity and composition profiles, U0 = 0.3 c_s, seeded
    white noise 1e-3 U0 on u_y; D_12 = 0.005).  Mole fractions run from 0.02
    to 0.98 rather than 0 to 1: in the tanh tails of pure bands a species
    falls to X ~ 1e-14 and the FP64 oracle drives it negative within a few
    steps (negative temperature by step 2-4 on a 6 x 256 x 6 grid), as with
    the trace species of the ternary tube.
  * ``random_mixture`` -- smooth random M-species field (sum of 16 Fourier
    modes per species), random molar masses and diffusivities.
  * ``ensemble_shapes`` / ``ensemble_domain`` -- the batched ensemble: 64
    ternary diffusion domains with edges uniform in 32..96, Dirichlet(1,1,1)
    left/right compositions and log-uniform diffusivities.
Common choices: T = 0.2 (inside the 0.2-0.5 range of Sec. 4.4); reference pressure P0 = T / m_mean with m_mean the
molar mass of the domain-mean composition (reference density 1);
mu_a = 0.1 P0, lambda_a = mu_a c_pa / 0.71
with c_pa = (cv_a + 1) R_U / m_a; cv_a = C-bar_{a,v}/R_U chosen by molar mass
(monatomic 3/2, diatomic 5/2, polyatomic 3).
"""

from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, Optional

import numpy as np

T_AMBIENT = 0.2
PR_TARGET = 0.71

_CV_BY_MASS = {2.0: 2.5, 4.0: 1.5, 16.0: 3.0, 28.0: 2.5, 40.0: 1.5, 44.0: 3.0}


def cv_for_mass(m: float) -> float:
    """Molar C_v / R_U by molecular identity of the molar mass."""
    return _CV_BY_MASS.get(float(m), 2.5)


@dataclass
class Workload:
    name: str
    molar_mass: np.ndarray        # (M,)
    cv_molar: np.ndarray          # (M,)
    D: np.ndarray                 # (M, M), diagonal 0 -> library default rule
    mu: np.ndarray                # (M,)
    lam: np.ndarray               # (M,)
    X: np.ndarray                 # (M, nz, ny, nx)
    u: np.ndarray                 # (3, nz, ny, nx)
    T: np.ndarray                 # (nz, ny, nx)
    P: np.ndarray                 # (nz, ny, nx)
    steps: int
    R_U: float = 1.0

    @property
    def M(self) -> int:
        return int(self.molar_mass.shape[0])

    @property
    def shape(self):
        return tuple(self.T.shape)

    @property
    def nodes(self) -> int:
        return int(np.prod(self.T.shape))

    def params(self, **overrides) -> Dict:
        d = dict(molar_mass=self.molar_mass.copy(), cv_molar=self.cv_molar.copy(),
                 D=self.D.copy(), mu=self.mu.copy(), lam=self.lam.copy(), R_U=self.R_U)
        d.update(overrides)
        return d


def _transport(molar_mass, cv_molar, P0, mu_factor):
    M = len(molar_mass)
    mu = np.full(M, mu_factor * P0)
    cp = (cv_molar + 1.0) / molar_mass
    lam = mu * cp / PR_TARGET
    return mu, lam


def _p0(X_mean, molar_mass, T):
    m_mean = float(np.dot(X_mean, molar_mass))
    return T / m_mean


def ternary_tube(nx: int = 64, ny: int = 4, nz: int = 4, steps: int = 1000,
                 width: float = 8.0, closed: bool = False) -> Workload:
    """Ternary H2/Ar/CH4 Loschmidt tube (Sec. 4.2): left half (0.5, 0.5, 0),
    right half (0.5, 0, 0.5), tanh steps of the given width.  Periodic (two
    steps, at the middle and across the periodic edge), or ``closed`` by walls
    normal to x (one step at the middle)."""
    mm = np.array([2.0, 40.0, 16.0])
    cv = np.array([cv_for_mass(m) for m in mm])
    D = np.array([[0.0, 0.05, 0.05], [0.05, 0.0, 0.01], [0.05, 0.01, 0.0]])
    XL = np.array([0.5, 0.5, 0.0])
    XR = np.array([0.5, 0.0, 0.5])
    x = np.arange(nx, dtype=np.float64)
    h = nx / 2.0
    if closed:
        s = 0.5 * (1.0 + np.tanh((x - (h - 0.5)) / width))
    else:
        # periodic double tanh step: right state on [h, nx), left on [0, h)
        s = 0.5 * (np.tanh((x - (h - 0.5)) / width) - np.tanh((x - (nx - 0.5)) / width)
                   - np.tanh((x + 0.5) / width) + 1.0)
    X = (1.0 - s)[None] * XL[:, None] + s[None] * XR[:, None]
    X = np.broadcast_to(X[:, None, None, :], (3, nz, ny, nx)).copy()
    X = X / X.sum(axis=0, keepdims=True)
    T = np.full((nz, ny, nx), T_AMBIENT)
    P0 = _p0(X.reshape(3, -1).mean(axis=1), mm, T_AMBIENT)
    P = np.full((nz, ny, nx), P0)
    u = np.zeros((3, nz, ny, nx))
    mu, lam = _transport(mm, cv, P0, 0.1)
    return Workload("ternary_tube", mm, cv, D, mu, lam, X, u, T, P, steps)


def acoustic_pulse(n: int = 128, x1: float = 0.5, amplitude: float = 1e-3, sigma: float = 6.0,
                   steps: int = 2000, shape: Optional[tuple] = None) -> Workload:
    mm = np.array([4.0, 40.0])
    cv = np.array([cv_for_mass(m) for m in mm])
    D = np.array([[0.0, 0.05], [0.05, 0.0]])
    nz, ny, nx = shape if shape is not None else (n, n, n)
    X = np.empty((2, nz, ny, nx))
    X[0] = x1
    X[1] = 1.0 - x1
    T = np.full((nz, ny, nx), T_AMBIENT)
    P0 = _p0(np.array([x1, 1.0 - x1]), mm, T_AMBIENT)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r2 = (x - nx / 2.0) ** 2 + (y - ny / 2.0) ** 2 + (z - nz / 2.0) ** 2
    P = P0 * (1.0 + amplitude * np.exp(-r2 / (2.0 * sigma ** 2)))
    u = np.zeros((3, nz, ny, nx))
    mu, lam = _transport(mm, cv, P0, 0.1)
    return Workload("acoustic_pulse", mm, cv, D, mu, lam, X, u, T, P, steps)


def shear_layer(n: int = 256, mach: float = 0.3, delta: float = 4.0, noise: float = 1e-3,
                seed: int = 1234, steps: int = 5000, shape: Optional[tuple] = None,
                floor: float = 0.02) -> Workload:
    mm = np.array([2.0, 28.0])
    cv = np.array([cv_for_mass(m) for m in mm])
    D = np.array([[0.0, 0.005], [0.005, 0.0]])
    nz, ny, nx = shape if shape is not None else (n, n, n)
    y = np.arange(ny, dtype=np.float64)
    y1, y2 = ny / 4.0, 3.0 * ny / 4.0
    band = 0.5 * (np.tanh((y - y1) / delta) - np.tanh((y - y2) / delta))   # 1 inside the band
    XA = floor + (1.0 - 2.0 * floor) * band      # no species falls to a trace
    X = np.empty((2, nz, ny, nx))
    X[0] = XA[None, :, None]
    X[1] = 1.0 - X[0]
    # reference sound speed of the 50/50 mixture (input recipe, Sec. 4.1 scaling)
    m50 = 0.5 * (mm[0] + mm[1])
    y50 = 0.5 * mm / m50
    cv50 = float(np.dot(y50, cv / mm))
    R50 = 1.0 / m50
    gamma50 = (cv50 + R50) / cv50
    U0 = mach * np.sqrt(gamma50 * R50 * T_AMBIENT)
    u = np.zeros((3, nz, ny, nx))
    u[0] = (U0 * (2.0 * band - 1.0))[None, :, None]
    rng = np.random.Generator(np.random.PCG64(seed))
    u[1] = noise * U0 * rng.uniform(-1.0, 1.0, size=(nz, ny, nx))
    T = np.full((nz, ny, nx), T_AMBIENT)
    P0 = _p0(np.array([0.5, 0.5]), mm, T_AMBIENT)
    P = np.full((nz, ny, nx), P0)
    mu, lam = _transport(mm, cv, P0, 0.1)
    return Workload("shear_layer", mm, cv, D, mu, lam, X, u, T, P, steps)


# The closed-tube cases of Sec. 4.2 (Eqs. ternaryConditions,
# ternaryConditionsCH4, ternaryConditionsH2): left / right mole fractions of
# H2, Ar, CH4.
LOSCHMIDT_CASES = {
    "1T": ([0.491, 0.509, 0.000], [0.000, 0.485, 0.515]),
    "2T": ([0.512, 0.000, 0.448], [0.000, 0.485, 0.515]),
    "3T": ([0.512, 0.000, 0.448], [0.491, 0.509, 0.000]),
}
# Binary diffusivities the section prints (1e-5 m^2/s): H2-Ar, H2-CH4, Ar-CH4.
LOSCHMIDT_D = (8.14543, 7.37433, 2.17321)


def loschmidt_tube(case: str = "1T", L: int = 96, width: float = 3.0, floor: float = 0.01,
                   D_h2_ar: float = 0.05, steps: int = 0) -> Workload:
    """The ternary Loschmidt tube of Sec. 4.2 (H2/Ar/CH4, molar masses 2.016,
    39.948, 16.043) on an L x 1 x 1 grid closed by walls at both x ends:
    the case's left and right compositions joined by a tanh step of the given
    width at the middle, every mole fraction floored at `floor` and the
    sides renormalised (a trace species left at zero drives the method
    unstable, as the design notes record).  The binary diffusivities keep
    the printed ratios, scaled so that D(H2, Ar) = D_h2_ar in lattice units.
    Uniform T and P, at rest."""
    XL, XR = (np.maximum(floor, np.asarray(v, dtype=np.float64)) for v in LOSCHMIDT_CASES[case])
    XL, XR = XL / XL.sum(), XR / XR.sum()
    mm = np.array([2.016, 39.948, 16.043])
    cv = np.array([2.5, 1.5, 3.0])
    d12, d13, d23 = (v * D_h2_ar / LOSCHMIDT_D[0] for v in LOSCHMIDT_D)
    D = np.array([[0.0, d12, d13], [d12, 0.0, d23], [d13, d23, 0.0]])
    x = np.arange(L, dtype=np.float64)
    s = 0.5 * (1.0 + np.tanh((x - (L / 2.0 - 0.5)) / width))
    X = ((1.0 - s)[None] * XL[:, None] + s[None] * XR[:, None]).reshape(3, 1, 1, L)
    T = np.full((1, 1, L), T_AMBIENT)
    P0 = _p0(X.reshape(3, -1).mean(axis=1), mm, T_AMBIENT)
    P = np.full((1, 1, L), P0)
    mu, lam = _transport(mm, cv, P0, 0.1)
    return Workload(f"loschmidt_{case}", mm, cv, D, mu, lam, X, np.zeros((3, 1, 1, L)), T, P, steps)


# Opposed jets of Sec. 4.3: H2, N2, O2, H2O; the jet compositions as printed
# (left, right).  Binary diffusivities: ratios of tabulated near-ambient
# values for these pairs (H2-N2 0.78, H2-O2 0.81, H2-H2O 0.92, N2-O2 0.21,
# N2-H2O 0.25, O2-H2O 0.25 cm^2/s), scaled in the recipe.
JETS_SPECIES = ("H2", "N2", "O2", "H2O")
JETS_MASS = np.array([2.016, 28.014, 31.998, 18.015])
JETS_CV = np.array([2.5, 2.5, 2.5, 3.0])
JETS_X = (np.array([0.1, 0.85, 0.0, 0.05]), np.array([0.0, 0.90, 0.1, 0.0]))
JETS_D_RATIO = np.array([[0.0, 0.78, 0.81, 0.92],
                         [0.78, 0.0, 0.21, 0.25],
                         [0.81, 0.21, 0.0, 0.25],
                         [0.92, 0.25, 0.25, 0.0]])


@dataclass
class JetInlets:
    """The two nozzles of the opposed-jets frame: interior rows [y0, y1) of
    both x faces, and for the nozzle at x = -1 (index 0) and at x = nx (1) the
    mole fractions, x velocity, temperature and pressure."""
    y0: int
    y1: int
    X: np.ndarray          # (2, M)
    u: np.ndarray          # (2,)
    T: np.ndarray          # (2,)
    P: np.ndarray          # (2,)


def opposed_jets(nx: int = 200, ny: int = 400, nz: int = 1, U: float = 0.01, floor: float = 0.01,
                 D_h2_n2: float = 0.02, mu_factor: float = 0.5, nozzle=(0.1, 0.9), steps: int = 40000):
    """Planar opposed jets of Sec. 4.3 on an nx x ny x nz interior (the paper:
    200 x 400 x 1).  Nozzles over the rows [0.1 ny, 0.9 ny) of both x faces;
    the jets' mole fractions as printed, floored at `floor` and renormalised
    (a species left at zero drives the method unstable, as for the Loschmidt
    tube); the left jet at x velocity U, the right one at the speed that
    gives equal momentum flux rho U^2 at the common T and P.  Binary
    diffusivities in the tabulated ratios with D(H2, N2) = D_h2_n2; species
    viscosities mu_factor * P0.  The interior starts at rest with the left
    composition for x < nx/2 and the right one beyond (a tanh step of 4
    cells).  Returns (Workload, JetInlets)."""
    XL, XR = (np.maximum(floor, v) for v in JETS_X)
    XL, XR = XL / XL.sum(), XR / XR.sum()
    mm, cv = JETS_MASS.copy(), JETS_CV.copy()
    M = 4
    T0 = T_AMBIENT
    P0 = _p0(0.5 * (XL + XR), mm, T0)
    mL, mR = float(XL @ mm), float(XR @ mm)
    UR = U * np.sqrt(mL / mR)                          # rho ~ m at equal T and P
    D = JETS_D_RATIO * (D_h2_n2 / JETS_D_RATIO[0, 1])
    mu, lam = _transport(mm, cv, P0, mu_factor)
    x = np.arange(nx) + 0.5
    s = 0.5 * (1.0 + np.tanh((x - 0.5 * nx) / 4.0))   # 0 left, 1 right
    X = np.empty((M, nz, ny, nx))
    for a in range(M):
        X[a] = (XL[a] + (XR[a] - XL[a]) * s)[None, None, :]
    u = np.zeros((3, nz, ny, nx))
    T = np.full((nz, ny, nx), T0)
    P = np.full((nz, ny, nx), P0)
    wl = Workload("opposed_jets", mm, cv, D, mu, lam, X, u, T, P, steps)
    y0, y1 = int(round(nozzle[0] * ny)), int(round(nozzle[1] * ny))
    inl = JetInlets(y0, y1, np.stack([XL, XR]), np.array([U, -UR]), np.array([T0, T0]), np.array([P0, P0]))
    return wl, inl


def with_frame(a):
    """A field (..., nz, ny, nx) on the grid with the one-node frame of the
    opposed-jets boundary set, (..., nz, ny + 2, nx + 2): the frame nodes
    take the nearest interior value (they are overwritten by the boundary
    rules before any population leaves them)."""
    a = np.asarray(a)
    pad = [(0, 0)] * (a.ndim - 2) + [(1, 1), (1, 1)]
    return np.pad(a, pad, mode="edge")


def khi_n2_h2o(shape=(200, 800, 800), reynolds: float = 11963.46, mach_r: float = 0.2, schmidt: float = 0.6,
               width: float = 0.0, steps: int = 0) -> Workload:
    """The three-dimensional Kelvin-Helmholtz instability of Sec. 4.5
    (Eqs. icKHI, uyKHI, uzKHI): N2 / H2O (molar masses 28.0134, 18.015;
    diatomic, polyatomic) on a periodic Lz x Ly x Lx grid (default
    200 x 800 x 800).  Three layers along y: X_H2O = 0.9 and u_x = +U for
    y < Ly/4 and y >= 3 Ly/4, X_H2O = 0.1 and u_x = -U between, with
    U = (mach_r / 2) c_s (relative Mach number mach_r, c_s of the 50/50
    mixture); u_y = 2U 0.01 sin(2 pi x / Lx), u_z = 2U 0.01 sin(2 pi z / Lz).
    The layers are sharp steps (width 0) or tanh steps of the given width.
    The species viscosity gives Re = 2 U Ly / nu in the bottom layer
    (nu = mu / rho, equal mu_a); the binary diffusivity D = nu / schmidt (the
    paper gives none); conductivities for Pr = 0.71.  Uniform T and P."""
    mm = np.array([28.0134, 18.015])
    cv = np.array([2.5, 3.0])
    nz, ny, nx = shape
    y = np.arange(ny, dtype=np.float64)
    if width > 0.0:
        outer = 1.0 - 0.5 * (np.tanh((y - ny / 4.0) / width) - np.tanh((y - 3.0 * ny / 4.0) / width))
    else:
        outer = ((y < ny / 4.0) | (y >= 3.0 * ny / 4.0)).astype(np.float64)
    xh2o = 0.1 + 0.8 * outer
    X = np.empty((2, nz, ny, nx))
    X[1] = xh2o[None, :, None]
    X[0] = 1.0 - X[1]
    m50 = 0.5 * (mm[0] + mm[1])
    y50 = 0.5 * mm / m50
    cv50 = float(np.dot(y50, cv / mm))
    gamma50 = (cv50 + 1.0 / m50) / cv50
    c50 = np.sqrt(gamma50 * T_AMBIENT / m50)
    U = 0.5 * mach_r * c50
    u = np.zeros((3, nz, ny, nx))
    u[0] = (U * (2.0 * outer - 1.0))[None, :, None]
    x = np.arange(nx, dtype=np.float64)
    z = np.arange(nz, dtype=np.float64)
    u[1] = (2.0 * U * 0.01 * np.sin(2.0 * np.pi * x / nx))[None, None, :]
    u[2] = (2.0 * U * 0.01 * np.sin(2.0 * np.pi * z / nz))[:, None, None]
    T = np.full((nz, ny, nx), T_AMBIENT)
    P0 = _p0(np.array([0.5, 0.5]), mm, T_AMBIENT)
    P = np.full((nz, ny, nx), P0)
    m_bottom = 0.1 * mm[0] + 0.9 * mm[1]
    rho_bottom = P0 * m_bottom / T_AMBIENT
    nu = 2.0 * U * ny / reynolds
    mu = np.full(2, nu * rho_bottom)
    lam = mu * (cv + 1.0) / mm / PR_TARGET
    D = np.array([[0.0, nu / schmidt], [nu / schmidt, 0.0]])
    return Workload("khi_n2_h2o", mm, cv, D, mu, lam, X, u, T, P, steps)


def variable_heats(molar_mass, seed: int = 0, T_ref: float = T_AMBIENT) -> np.ndarray:
    """Synthetic temperature-dependent molar heats for Sec. 3.1 (no
    thermochemical data exist here): C-bar_{a,v}(T) / R_U = c0 + c1 T + c2 T^2
    per species, with the value at T_ref the molecular-identity constant of
    cv_for_mass and slopes drawn from `seed` so the heat changes by -10 % ..
    +40 % between T = 0 and 2 T_ref while staying positive.  Returns (M, 3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for m in np.asarray(molar_mass, dtype=np.float64):
        c_ref = cv_for_mass(float(m))
        s1, s2 = rng.uniform(-0.05, 0.2), rng.uniform(0.0, 0.1)       # fractional changes per T_ref, per T_ref^2
        c1, c2 = s1 * c_ref / T_ref, s2 * c_ref / T_ref ** 2
        out.append([c_ref - c1 * T_ref - c2 * T_ref ** 2, c1, c2])
    return np.array(out)


def random_mixture(M: int = 8, n: int = 192, seed: int = 7, steps: int = 3000,
                   shape: Optional[tuple] = None, modes: int = 16, velocity: float = 0.0,
                   field_seed: Optional[int] = None, amplitude: float = 0.5) -> Workload:
    """Species constants (molar masses, C_v, diffusivities) from `seed`; the
    initial fields from `field_seed` (default: the same generator, so one
    seed fixes everything), so one mixture can be drawn in many states.
    Mole fractions are max(0.05, 1 + amplitude * phi) renormalised, with phi
    the normalised sum of Fourier modes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nz, ny, nx = shape if shape is not None else (n, n, n)
    mm = rng.uniform(2.0, 44.0, size=M)
    cv = rng.choice(np.array([1.5, 2.5, 3.0]), size=M)
    D = np.zeros((M, M))
    for a in range(M):
        for b in range(a + 1, M):
            D[a, b] = D[b, a] = float(np.exp(rng.uniform(np.log(0.005), np.log(0.1))))
    if M == 1:
        D[0, 0] = 0.05
    if field_seed is not None:
        rng = np.random.Generator(np.random.PCG64(field_seed))
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    Xt = np.empty((M, nz, ny, nx))
    for a in range(M):
        phi = np.zeros((nz, ny, nx))
        for _ in range(modes):
            kx, ky, kz = rng.integers(-3, 4, size=3)
            A = rng.uniform(0.0, 1.0)
            ps = rng.uniform(0.0, 2.0 * np.pi)
            phi += A * np.cos(2.0 * np.pi * (kx * x / nx + ky * y / ny + kz * z / nz) + ps)
        mx = np.abs(phi).max()
        phi = phi / mx if mx > 0 else phi
        Xt[a] = np.maximum(0.05, 1.0 + amplitude * phi)
    X = Xt / Xt.sum(axis=0, keepdims=True)
    T = np.full((nz, ny, nx), T_AMBIENT)
    P0 = _p0(X.reshape(M, -1).mean(axis=1), mm, T_AMBIENT)
    P = np.full((nz, ny, nx), P0)
    u = np.zeros((3, nz, ny, nx))
    if velocity > 0.0:
        u = velocity * rng.uniform(-1.0, 1.0, size=(3, nz, ny, nx))
    mu, lam = _transport(mm, cv, P0, 0.1)
    return Workload("random_mixture", mm, cv, D, mu, lam, X, u, T, P, steps)


def ensemble_shapes(ndomains: int = 64, seed: int = 4, lo: int = 32, hi: int = 96):
    """Grid shapes (nz, ny, nx) of the batched ensemble, each edge uniform in
    lo..hi (mean domain about 3.3e5 nodes at the defaults)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [tuple(int(v) for v in rng.integers(lo, hi + 1, size=3)) for _ in range(ndomains)]


def ensemble_domain(shape, seed: int, steps: int = 2000, width: float = 8.0,
                    floor: float = 0.02) -> Workload:
    """One ternary diffusion domain of the ensemble: m = 2, 40, 16, symmetric
    D_ab log-uniform in [0.005, 0.1], left/right mole fractions drawn from
    Dirichlet(1, 1, 1) (floored at `floor` and renormalised, so no species is
    a trace in the tanh tails) joined by periodic tanh steps along x of scale
    `width` (8 cells, as the ternary tube), uniform T and P, at rest."""
    nz, ny, nx = shape
    rng = np.random.Generator(np.random.PCG64(seed))
    mm = np.array([2.0, 40.0, 16.0])
    cv = np.array([cv_for_mass(m) for m in mm])
    D = np.zeros((3, 3))
    for a in range(3):
        for b in range(a + 1, 3):
            D[a, b] = D[b, a] = float(np.exp(rng.uniform(np.log(0.005), np.log(0.1))))
    XL, XR = (np.maximum(rng.dirichlet(np.ones(3)), floor) for _ in range(2))
    XL, XR = XL / XL.sum(), XR / XR.sum()
    x = np.arange(nx, dtype=np.float64)
    h = nx / 2.0
    s = 0.5 * (np.tanh((x - (h - 0.5)) / width) - np.tanh((x - (nx - 0.5)) / width)
               - np.tanh((x + 0.5) / width) + 1.0)
    X = (1.0 - s)[None] * XL[:, None] + s[None] * XR[:, None]
    X = np.broadcast_to(X[:, None, None, :], (3, nz, ny, nx)).copy()
    X = X / X.sum(axis=0, keepdims=True)
    T = np.full((nz, ny, nx), T_AMBIENT)
    P0 = _p0(X.reshape(3, -1).mean(axis=1), mm, T_AMBIENT)
    P = np.full((nz, ny, nx), P0)
    u = np.zeros((3, nz, ny, nx))
    mu, lam = _transport(mm, cv, P0, 0.1)
    return Workload("ensemble_domain", mm, cv, D, mu, lam, X, u, T, P, steps)


def perturbation(shape, scale: float, seed: int) -> np.ndarray:
    """Seeded multiplicative noise (1 + scale * U(-1, 1)) used by tests to move
    a state off equilibrium; drawn here so both sides see the same numbers."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return 1.0 + scale * rng.uniform(-1.0, 1.0, size=shape)


def slaved_species(wl: Workload) -> int:
    """Strong-coupling choice of the slaved species (Sec. 3.5.2 advises the one
    carrying most mass): the species whose SMALLEST mass fraction over the
    initial field is largest, so that no node slaves a vanishing species."""
    mm = wl.molar_mass.reshape((wl.M,) + (1,) * len(wl.shape))
    Y = wl.X * mm
    Y = Y / Y.sum(axis=0, keepdims=True)
    return int(np.argmax(Y.reshape(wl.M, -1).min(axis=1)))


def closure_initial_weights(M: int, seed: int = 0, hidden: int = 128) -> np.ndarray:
    """Seeded initial weights of the closure network, packed W1 [H][F] | b1 |
    W2 [H][H] | b2 | W3 [O][H] | b3 (F = pad16(4M + M(M-1)/2 + 1), O =
    pad16(3M)): uniform in +-sqrt(6 / fan_in) (He), zero biases, and zero
    rows of W3 on the padded outputs."""
    def pad16(n):
        return (n + 15) // 16 * 16
    F, O = pad16(4 * M + M * (M - 1) // 2 + 1), pad16(3 * M)
    rng = np.random.Generator(np.random.PCG64(seed))
    W1 = rng.uniform(-1, 1, (hidden, F)) * np.sqrt(6.0 / F)
    W2 = rng.uniform(-1, 1, (hidden, hidden)) * np.sqrt(6.0 / hidden)
    W3 = rng.uniform(-1, 1, (O, hidden)) * np.sqrt(6.0 / hidden) * 0.1
    W3[3 * M:] = 0.0
    parts = [W1, np.zeros(hidden), W2, np.zeros(hidden), W3, np.zeros(O)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)
