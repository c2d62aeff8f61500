"""FP64 oracle of the learned Stefan-Maxwell closure: the per-node features,
the exact targets, the small network (forward, backward, loss) and one Adam
step.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.

What is learned.  At every node the species velocities come from one M x M
linear system with three right-hand sides (Eq. transform12, written for the
fluxes J_a = rho_a V_a):

    J_a + (1/2) sum_{b != a} (1/tau_ab) (Y_b J_a - Y_a J_b) = r_a,
    r_a = j_a - rho_a u,

with 1/tau_ab from Eq. (tauab).  The network replaces that solve.  Its
interface (a convention that the CUDA path writes independently):

  * s = max_{a,c} |r_a,c| normalises the right-hand side (s = 0 gives J = 0);
  * features, F = pad16(M + 3M + M(M-1)/2 + 1) values per node:
      [0, M)                  the mole fractions X_a (Eq. moleFractionDefinition),
      [M, 4M)                 r_a,c / s at M + 3a + c,
      [4M, 4M + M(M-1)/2)     h_ab / (1 + h_ab) for the pairs a < b in
                              lexicographic order, h_ab = (1/2)(1/tau_ab)(Y_a + Y_b),
      4M + M(M-1)/2           the constant 1,
      the rest                0;
  * outputs, O = pad16(3M) values: the correction J_a,c / s - J0_a,c at
    3a + c to the one-sweep Jacobi estimate J0_a,c = (r_a,c / s) / A_aa (A
    the matrix of the system below), the rest unused -- the network learns
    what the diagonal misses, a smaller quantity than J itself, so the bf16
    rounding of its activations costs proportionally less;
  * the network: two hidden layers of width H = 128 with the exact GELU,
    x Phi(x) = x (1 + erf(x / sqrt 2)) / 2, and a linear output layer;
  * weights are packed as W1 [H][F], b1 [H], W2 [H][H], b2 [H], W3 [O][H],
    b3 [O] (row-major, FP32 in the library);
  * the loss is the mean of (out - target)^2 over the samples and the 3M
    valid outputs.

The closure is accepted at a node when the residual of the system for the
network's fluxes, max_{a,c} |(A J~)_a,c - r_a,c / s| with J~ = J0 + output,
is within a bound; elsewhere the exact solve is used.
"""

from __future__ import annotations

import math

import numpy as np

from .lbm_oracle import Params, inv_tau_ab

H = 128


def _pad16(n: int) -> int:
    return (n + 15) // 16 * 16


def closure_dims(M: int):
    """(F, O, number of pair features) for M species."""
    npair = M * (M - 1) // 2
    return _pad16(M + 3 * M + npair + 1), _pad16(3 * M), npair


def weight_count(M: int) -> int:
    F, O, _ = closure_dims(M)
    return H * F + H + H * H + H + O * H + O


def unpack(w, M: int):
    """Split a packed weight vector into (W1, b1, W2, b2, W3, b3)."""
    F, O, _ = closure_dims(M)
    w = np.asarray(w, dtype=np.float64)
    sizes = [(H, F), (H,), (H, H), (H,), (O, H), (O,)]
    out, k = [], 0
    for s in sizes:
        n = int(np.prod(s))
        out.append(w[k:k + n].reshape(s))
        k += n
    assert k == w.size, (k, w.size)
    return out


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def sm_system(st, prm: Params, itab=None):
    """The J-form matrix A[n, M, M] of Eq. (transform12) and the right-hand
    sides r[n, M, 3] at every node (nodes flattened)."""
    M = prm.M
    if itab is None:
        itab = inv_tau_ab(st, prm)
    Y = st["Y"]
    n = int(np.prod(st["T"].shape)) if st["T"].shape else 1
    A = np.zeros((n, M, M))
    for a in range(M):
        diag = np.ones(n)
        for b in range(M):
            if b != a:
                diag = diag + 0.5 * (itab[a, b] * Y[b]).reshape(n)
                A[:, a, b] = (-0.5 * itab[a, b] * Y[a]).reshape(n)
        A[:, a, a] = diag
    r = (st["j_a"] - st["rho_a"][:, None] * st["u_sp"][None]).reshape(M, 3, n).transpose(2, 0, 1)
    return A, r


def features_and_targets(st, prm: Params):
    """Features [n, F], exact normalised targets [n, O], the scale s [n], and
    the system (A, r), at every node of a node_state."""
    M = prm.M
    F, O, npair = closure_dims(M)
    itab = inv_tau_ab(st, prm)
    A, r = sm_system(st, prm, itab)
    n = A.shape[0]
    s = np.abs(r).reshape(n, -1).max(axis=1)
    inv_s = np.where(s > 0, 1.0 / np.where(s > 0, s, 1.0), 0.0)
    rn = r * inv_s[:, None, None]
    feat = np.zeros((n, F))
    X = st["X"].reshape(M, n)
    Y = st["Y"].reshape(M, n)
    feat[:, :M] = X.T
    feat[:, M:4 * M] = rn.reshape(n, 3 * M)
    k = 4 * M
    for a in range(M):
        for b in range(a + 1, M):
            h = 0.5 * itab[a, b].reshape(n) * (Y[a] + Y[b])
            feat[:, k] = h / (1.0 + h)
            k += 1
    feat[:, k] = 1.0
    J = np.linalg.solve(A, rn)                                   # exact normalised fluxes
    tgt = np.zeros((n, O))
    tgt[:, :3 * M] = (J - jacobi_estimate(A, rn)).reshape(n, 3 * M)
    return feat, tgt, s, A, r


def jacobi_estimate(A, rn):
    """J0_a,c = rn_a,c / A_aa (one Jacobi sweep from zero)."""
    d = np.einsum("naa->na", A)
    return rn / d[:, :, None]


def gelu(x):
    """Exact GELU, x Phi(x) with the standard normal CDF Phi."""
    from scipy.special import erf
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(w, feat, M: int):
    """Network output [n, O] and the pre-activations of the two hidden layers."""
    W1, b1, W2, b2, W3, b3 = unpack(w, M)
    h1 = feat @ W1.T + b1
    a1 = gelu(h1)
    h2 = a1 @ W2.T + b2
    a2 = gelu(h2)
    out = a2 @ W3.T + b3
    return out, (h1, a1, h2, a2)


def loss(w, feat, tgt, M: int) -> float:
    out, _ = forward(w, feat, M)
    d = out[:, :3 * M] - tgt[:, :3 * M]
    return float((d * d).sum() / d.size)


def gradients(w, feat, tgt, M: int):
    """d loss / d w, packed like w, by the chain rule through the three layers."""
    W1, b1, W2, b2, W3, b3 = unpack(w, M)
    out, (h1, a1, h2, a2) = forward(w, feat, M)
    n = feat.shape[0]
    dout = np.zeros_like(out)
    dout[:, :3 * M] = 2.0 * (out[:, :3 * M] - tgt[:, :3 * M]) / (n * 3 * M)
    gW3 = dout.T @ a2
    gb3 = dout.sum(axis=0)
    dh2 = (dout @ W3) * gelu_grad(h2)
    gW2 = dh2.T @ a1
    gb2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * gelu_grad(h1)
    gW1 = dh1.T @ feat
    gb1 = dh1.sum(axis=0)
    return pack([gW1, gb1, gW2, gb2, gW3, gb3])


def adam_step(w, g, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) at step t >= 1;
    returns the new (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def residual(A, r, s, out, M: int):
    """max_{a,c} |(A J~)_a,c - r_a,c / s| per node, J~ = J0 + the output."""
    n = A.shape[0]
    inv_s = np.where(s > 0, 1.0 / np.where(s > 0, s, 1.0), 0.0)
    rn = r * inv_s[:, None, None]
    Jn = jacobi_estimate(A, rn) + out[:, :3 * M].reshape(n, M, 3)
    res = np.einsum("nab,nbc->nac", A, Jn) - rn
    return np.abs(res).reshape(n, -1).max(axis=1)
