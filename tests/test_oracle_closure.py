"""Pins of the oracle of the learned Stefan-Maxwell closure (no GPU): the
exact targets against the binary closed form of Eq. (transform12), the
feature layout, the network against networks whose output is known in closed
form, the backward pass against central finite differences, and Adam's first
step against its known sign property."""

import math

import numpy as np
import pytest

import oracle as O
from oracle import closure as CL

from test_oracle_pins import _rand_params, _rand_state


def _state(M, shape=(3, 4, 5), seed=3, coupling="strong"):
    prm = _rand_params(M, coupling=coupling, seed=seed)
    pops = _rand_state(prm, shape, seed=seed + 1)
    st = O.node_state(O.moments(pops, prm), prm)
    return prm, st


def test_dims_and_packing():
    for M, F, Out in ((2, 16, 16), (3, 16, 16), (4, 32, 16), (8, 64, 32)):
        f, o, npair = CL.closure_dims(M)
        assert (f, o, npair) == (F, Out, M * (M - 1) // 2)
        assert M + 3 * M + npair + 1 <= f
        w = np.arange(CL.weight_count(M), dtype=float)
        np.testing.assert_array_equal(CL.pack(CL.unpack(w, M)), w)


def test_gelu_values_and_odd_identity():
    # GELU(x) = x Phi(x): Phi(0) = 1/2, Phi(1) = 0.8413447460685429 (standard
    # normal table); GELU(x) - GELU(-x) = x because Phi(x) + Phi(-x) = 1.
    assert CL.gelu(np.array(0.0)) == 0.0
    assert abs(CL.gelu(np.array(1.0)) - 0.8413447460685429) < 1e-15
    assert abs(CL.gelu(np.array(-1.0)) + (1 - 0.8413447460685429)) < 1e-15
    x = np.linspace(-6, 6, 101)
    np.testing.assert_allclose(CL.gelu(x) - CL.gelu(-x), x, atol=1e-14)
    h = 1e-6
    np.testing.assert_allclose(CL.gelu_grad(x), (CL.gelu(x + h) - CL.gelu(x - h)) / (2 * h), atol=1e-8)


def test_binary_targets_closed_form():
    # M = 2 under strong coupling: r_1 + r_2 = 0, so Eq. (transform12) gives
    # J_1 = -J_2 = r_1 / (1 + (1/2)(1/tau_12)(Y_1 + Y_2)) = r_1 / (1 + 1/(2 tau_12)).
    prm, st = _state(2)
    feat, tgt, s, A, r = CL.features_and_targets(st, prm)
    itab = O.lbm_oracle.inv_tau_ab(st, prm)[0, 1].ravel()
    np.testing.assert_allclose(r[:, 0, :] + r[:, 1, :], 0, atol=1e-15)
    J1 = r[:, 0, :] / (1.0 + 0.5 * itab)[:, None] / s[:, None]
    # targets are the corrections to the Jacobi estimate r_a / (s A_aa), with
    # A_11 = 1 + itab_12 Y_2 / 2 and A_22 = 1 + itab_12 Y_1 / 2
    Y = st["Y"].reshape(2, -1)
    J0_1 = r[:, 0, :] / s[:, None] / (1.0 + 0.5 * itab * Y[1])[:, None]
    J0_2 = r[:, 1, :] / s[:, None] / (1.0 + 0.5 * itab * Y[0])[:, None]
    np.testing.assert_allclose(tgt[:, 0:3], J1 - J0_1, rtol=0, atol=1e-12)   # |targets| <= 1
    np.testing.assert_allclose(tgt[:, 3:6], -J1 - J0_2, rtol=0, atol=1e-12)
    assert np.all(tgt[:, 6:] == 0)
    # feature layout: X_a, r / s, h_12 / (1 + h_12) with h_12 = itab_12 / 2, 1, zeros
    np.testing.assert_allclose(feat[:, 0:2], st["X"].reshape(2, -1).T, rtol=1e-15)
    np.testing.assert_allclose(feat[:, 2:8], r.reshape(-1, 6) / s[:, None], rtol=1e-15)
    np.testing.assert_allclose(np.abs(feat[:, 2:8]).max(axis=1), 1.0, rtol=2e-16)
    h = 0.5 * itab
    np.testing.assert_allclose(feat[:, 8], h / (1 + h), rtol=1e-15)
    assert np.all(feat[:, 9] == 1.0) and np.all(feat[:, 10:] == 0)


@pytest.mark.parametrize("M", [3, 8])
def test_targets_solve_the_system(M):
    prm, st = _state(M, coupling="weak" if M == 3 else "strong")
    feat, tgt, s, A, r = CL.features_and_targets(st, prm)
    assert np.all(CL.residual(A, r, s, tgt, M) < 1e-13)
    n = A.shape[0]
    Jn = tgt[:, :3 * M].reshape(n, M, 3) + CL.jacobi_estimate(A, r / s[:, None, None])
    # sum_a J_a = 0 when sum_a r_a = 0 (columns of A - I sum to zero)
    if prm.coupling == "strong":
        np.testing.assert_allclose(Jn.sum(axis=1), 0, atol=1e-13)
    # the species velocities of the oracle's own solve are J_a / rho_a
    V = O.sm_momenta(st, prm)
    J = Jn * s[:, None, None]
    np.testing.assert_allclose(J.transpose(1, 2, 0).reshape(V.shape),
                               V * st["rho_a"][:, None], rtol=1e-9, atol=1e-14)


def _identity_net(M, shift=0.37, perm_seed=0):
    """Weights with out[k] = feat[sigma(k)] for every output k: layer 1 makes
    (x + t, -x - t), layer 2 GELU(x+t) - GELU(-x-t) - t = x and its negative,
    layer 3 the difference again.  Every bias and weight enters."""
    F, Out, _ = CL.closure_dims(M)
    H = CL.H
    assert 2 * F <= H
    sigma = np.random.Generator(np.random.PCG64(perm_seed)).permutation(F)[:Out]
    W1 = np.zeros((H, F)); b1 = np.zeros(H)
    for j in range(F):
        W1[j, j] = 1.0; b1[j] = shift
        W1[F + j, j] = -1.0; b1[F + j] = -shift
    W2 = np.zeros((H, H)); b2 = np.zeros(H)
    for j in range(F):
        W2[j, j] = 1.0; W2[j, F + j] = -1.0; b2[j] = -shift
        W2[F + j, j] = -1.0; W2[F + j, F + j] = 1.0; b2[F + j] = shift
    W3 = np.zeros((Out, H)); b3 = np.full(Out, 0.25)
    for k in range(Out):
        W3[k, sigma[k]] = 1.0; W3[k, F + sigma[k]] = -1.0
    return CL.pack([W1, b1, W2, b2, W3, b3]), sigma


@pytest.mark.parametrize("M", [2, 8])
def test_forward_identity_network(M):
    F, Out, _ = CL.closure_dims(M)
    w, sigma = _identity_net(M)
    x = np.random.Generator(np.random.PCG64(5)).uniform(-2, 2, (40, F))
    out, _ = CL.forward(w, x, M)
    np.testing.assert_allclose(out, x[:, sigma] + 0.25, atol=1e-13)


def test_gradients_match_finite_differences():
    M = 3
    F, Out, _ = CL.closure_dims(M)
    rng = np.random.Generator(np.random.PCG64(11))
    w = rng.normal(0, 0.3, CL.weight_count(M))
    x = rng.uniform(-1, 1, (7, F))
    t = rng.uniform(-1, 1, (7, Out))
    g = CL.gradients(w, x, t, M)
    # every block of the packed vector, including padded outputs (zero)
    W1, b1, W2, b2, W3, b3 = CL.unpack(g, M)
    assert np.all(W3[3 * M:] == 0) and np.all(b3[3 * M:] == 0)
    idx = rng.choice(w.size, 60, replace=False)
    h = 1e-6
    for k in idx:
        wp = w.copy(); wp[k] += h
        wm = w.copy(); wm[k] -= h
        fd = (CL.loss(wp, x, t, M) - CL.loss(wm, x, t, M)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(fd)), (k, fd, g[k])
    assert CL.loss(w, x, CL.forward(w, x, M)[0], M) == 0.0


def test_adam_first_step_is_lr_times_sign():
    # From m = v = 0 the bias-corrected ratio m^/sqrt(v^) is g/|g|.
    rng = np.random.Generator(np.random.PCG64(2))
    w = rng.normal(size=50)
    g = rng.normal(size=50)
    w1, m, v = CL.adam_step(w, g, np.zeros(50), np.zeros(50), 1, lr=1e-3, eps=0.0)
    np.testing.assert_allclose(w1, w - 1e-3 * np.sign(g), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-12)
