"""Linearised Maxwell-Stefan diffusion in a closed tube (textbook theory, not
the lattice Boltzmann method): the reference the osmotic-diffusion tests
compare the method's half-tube averages with (Sec. 4.2 compares its ternary
tube with such a theory).

For an ideal gas at uniform temperature and pressure the molar fluxes
relative to the molar-average velocity are J = -c [D] grad X for species
1..n-1, [D] = [B]^-1 with
    B_ii = X_i / D_in + sum_{k != i} X_k / D_ik,
    B_ij = -X_i (1 / D_ij - 1 / D_in)       (i != j),
and in a closed tube the molar-average velocity vanishes, so
dX/dt = [D] d^2X/dx^2.  Linearised at the mean composition, each cosine
mode cos(m pi (x + 1/2) / L) of the walls' Neumann problem decays as
exp(-[D] (m pi / L)^2 t)."""

import numpy as np


def fick_matrix(Xbar, D):
    M = len(Xbar)
    n = M - 1
    B = np.zeros((n, n))
    for i in range(n):
        B[i, i] = Xbar[i] / D[i, n] + sum(Xbar[k] / D[i, k] for k in range(M) if k != i)
        for j in range(n):
            if j != i:
                B[i, j] = -Xbar[i] * (1.0 / D[i, j] - 1.0 / D[i, n])
    return np.linalg.inv(B)


def half_tube_differences(X0, D, times):
    """Left-half minus right-half mean mole fraction of every species at each
    time, for the initial profile X0 (M, L) between walls at x = -1/2 and
    L - 1/2."""
    M, L = X0.shape
    Xbar = X0.mean(axis=1)
    lam, V = np.linalg.eig(fick_matrix(Xbar, D))
    Vi = np.linalg.inv(V)
    x = np.arange(L)
    out = []
    for t in times:
        X = np.repeat(Xbar[:M - 1, None], L, axis=1).astype(complex)
        for m in range(1, L):
            c = np.cos(m * np.pi * (x + 0.5) / L)
            a0 = (X0[:M - 1] - Xbar[:M - 1, None]) @ c * 2.0 / L
            am = V @ (np.exp(-lam * (m * np.pi / L) ** 2 * t) * (Vi @ a0))
            X = X + am[:, None] * c[None, :]
        X = X.real
        full = np.vstack([X, 1.0 - X.sum(axis=0, keepdims=True)])
        out.append(full[:, :L // 2].mean(axis=1) - full[:, L // 2:].mean(axis=1))
    return np.array(out)


def osmotic_tube(L, width=4.0):
    """H2/Ar/CH4 (m = 2, 40, 16) tube: hydrogen at the same mole fraction in
    both halves, argon and methane exchanged; D_12 != D_13 couples hydrogen to
    their gradients.  Returns (X0 (3, L), D)."""
    D = np.array([[0.0, 0.05, 0.02], [0.05, 0.0, 0.01], [0.02, 0.01, 0.0]])
    x = np.arange(L, dtype=float)
    s = 0.5 * (1.0 + np.tanh((x - (L / 2 - 0.5)) / width))
    XL, XR = np.array([0.4, 0.35, 0.25]), np.array([0.4, 0.25, 0.35])
    return (1.0 - s)[None] * XL[:, None] + s[None] * XR[:, None], D
