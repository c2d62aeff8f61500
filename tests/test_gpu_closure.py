"""The learned Stefan-Maxwell closure on the GPU (through the C ABI) against
the FP64 oracle of oracle/closure.py: the training pairs the method generates,
the tensor-core network, the training kernels' gradients and Adam step, and
the step with the network in place of the solve (exact fallback)."""

import numpy as np
import pytest

import oracle as O
from oracle import closure as CL
from paper_2004_11286_gb300 import workloads as W

from gpu_helpers import field_errors, gpu_handle, oracle_params, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2004_11286_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()


def _bf16(x):
    """Round-to-nearest-even to bf16, returned as float64 (test-side model of
    the tensor-core operand rounding)."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32)
    r = ((a >> 16) & 1) + np.uint32(0x7FFF)
    return ((a + r) & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)


def _cuda(a, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float32, device="cuda")


def _state(M, shape, seed, coupling="strong", precision="fp64"):
    wl = W.random_mixture(M=M, shape=shape, seed=seed, velocity=0.03)
    prm = oracle_params(wl, coupling=coupling)
    pops = O.init_populations(wl.X, wl.u, wl.T, wl.P, prm) * W.perturbation((M + 2, 27) + shape, 0.01, seed)
    h = gpu_handle(wl, precision, coupling=coupling)
    h.set_populations(pops)
    return wl, prm, pops, h


# ---------------------------------------------------------------------------
# Training pairs: features and exact targets at every node.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("M,coupling,precision", [(2, "strong", "fp64"), (3, "weak", "fp64"),
                                                  (8, "strong", "fp64"), (8, "strong", "fp32")])
def test_samples_match_oracle(M, coupling, precision):
    wl, prm, pops, h = _state(M, (3, 5, 7), 60 + M, coupling, precision)
    feat, tgt = h.closure_samples()
    st = O.node_state(O.moments(pops, prm), prm)
    of, ot, s, A, r = CL.features_and_targets(st, prm)
    f, t = feat.cpu().numpy(), tgt.cpu().numpy()
    if precision == "fp64":                                # FP32 rounding of the outputs only
        assert np.abs(f - of).max() < 2e-7
        assert np.abs(t - ot).max() < 2e-6
    else:
        # r_a = j_a - rho_a u cancels: its FP32 error is eps |rho_a u|, which
        # is up to ~1e3 eps in units of s = max|r| on these states
        rcols = slice(M, 4 * M)
        other = np.ones(f.shape[1], bool)
        other[rcols] = False
        assert np.abs(f[:, other] - of[:, other]).max() < 2e-6
        assert np.abs(f[:, rcols] - of[:, rcols]).max() < 1e-3
        assert np.abs(t - ot).max() < 1e-3
    h.close()


# ---------------------------------------------------------------------------
# The tensor-core network (bf16 operands, FP32 accumulation).
# ---------------------------------------------------------------------------
def _identity_net(M, shift=0.375):
    F, Out, _ = CL.closure_dims(M)
    H = CL.H
    sigma = np.random.Generator(np.random.PCG64(1)).permutation(F)[:Out]
    W1 = np.zeros((H, F)); b1 = np.zeros(H)
    W2 = np.zeros((H, H)); b2 = np.zeros(H)
    for j in range(F):
        W1[j, j], b1[j], W1[F + j, j], b1[F + j] = 1.0, shift, -1.0, -shift
        W2[j, j], W2[j, F + j], b2[j] = 1.0, -1.0, -shift
        W2[F + j, j], W2[F + j, F + j], b2[F + j] = -1.0, 1.0, shift
    W3 = np.zeros((Out, H)); b3 = np.full(Out, 0.25)
    for k in range(Out):
        W3[k, sigma[k]], W3[k, F + sigma[k]] = 1.0, -1.0
    return CL.pack([W1, b1, W2, b2, W3, b3]), sigma


@pytest.mark.parametrize("M", [2, 4, 8])
def test_forward_identity_network(M):
    # out[k] = x[sigma(k)] + 1/4 exactly in real arithmetic; a transposed or
    # misplaced operand, a wrong descriptor stride or a lost bias gives O(1)
    # errors, the bf16 rounding of inputs and activations stays below 2e-2.
    F, Out, _ = CL.closure_dims(M)
    _, _, _, h = _state(M, (2, 2, 2), 5, precision="fp32")
    w, sigma = _identity_net(M)
    h.set_closure_weights(w)
    n = 1000                                  # several tiles and a ragged tail
    x = np.random.Generator(np.random.PCG64(2)).uniform(-2, 2, (n, F)).astype(np.float32)
    out = h.closure_forward(_cuda(x)).cpu().numpy()
    ref = _bf16(x)[:, sigma] + 0.25
    assert np.abs(out - ref).max() < 2e-2
    h.close()


@pytest.mark.parametrize("M", [3, 8])
def test_forward_random_network_matches_oracle(M):
    F, Out, nw = CL.closure_dims(M)[0], CL.closure_dims(M)[1], CL.weight_count(M)
    _, _, _, h = _state(M, (2, 2, 2), 6, precision="fp32")
    w = W.closure_initial_weights(M, seed=3)
    w[CL.unpack(np.arange(nw), M)[5].astype(int)] = 0.1   # nonzero output biases
    h.set_closure_weights(w)
    n = 517
    x = np.random.Generator(np.random.PCG64(4)).uniform(-1, 1, (n, F)).astype(np.float32)
    out = h.closure_forward(_cuda(x)).cpu().numpy()
    parts = CL.unpack(w.astype(np.float64), M)
    wq = CL.pack([_bf16(p) if k in (0, 2, 4) else p for k, p in enumerate(parts)])
    ref, _ = CL.forward(wq, _bf16(x), M)
    # the remaining gap is the bf16 rounding of the two hidden activations
    assert rel(out[:, :3 * M], ref[:, :3 * M]) < 2e-2
    h.close()


# ---------------------------------------------------------------------------
# Training kernels: gradient and Adam step against the oracle.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("M", [3, 8])
def test_gradients_match_oracle(M):
    F, Out, _ = CL.closure_dims(M)
    _, _, _, h = _state(M, (2, 2, 2), 7, precision="fp32")
    rng = np.random.Generator(np.random.PCG64(8))
    w = W.closure_initial_weights(M, seed=5)
    h.set_closure_weights(w)
    n = 300
    x = rng.uniform(-1, 1, (n, F)).astype(np.float32)
    t = rng.uniform(-1, 1, (n, Out)).astype(np.float32)
    loss, g = h.closure_loss_grad(_cuda(x), _cuda(t))
    g = g.cpu().numpy()
    w64 = w.astype(np.float64)
    og = CL.gradients(w64, x.astype(np.float64), t.astype(np.float64), M)
    ol = CL.loss(w64, x.astype(np.float64), t.astype(np.float64), M)
    assert abs(loss - ol) <= 1e-5 * ol
    for blk, (a, b) in enumerate(zip(CL.unpack(g, M), CL.unpack(og, M))):
        assert np.abs(a - b).max() <= 1e-4 * max(np.abs(b).max(), 1e-12), blk
    h.close()


def test_adam_step_matches_oracle():
    M = 3
    F, Out, _ = CL.closure_dims(M)
    _, _, _, h = _state(M, (2, 2, 2), 9, precision="fp32")
    rng = np.random.Generator(np.random.PCG64(10))
    w = W.closure_initial_weights(M, seed=6)
    h.set_closure_weights(w)
    n = 200
    x = rng.uniform(-1, 1, (n, F)).astype(np.float32)
    t = rng.uniform(-1, 1, (n, Out)).astype(np.float32)
    w64 = w.astype(np.float64)
    g = CL.gradients(w64, x.astype(np.float64), t.astype(np.float64), M)
    w1, m, v = CL.adam_step(w64, g, np.zeros_like(g), np.zeros_like(g), 1, lr=1e-3)
    g2 = CL.gradients(w1, x.astype(np.float64), t.astype(np.float64), M)
    w2, _, _ = CL.adam_step(w1, g2, m, v, 2, lr=1e-3)
    h.closure_train(_cuda(x), _cuda(t), batch=n, steps=2, lr=1e-3)
    got = h.closure_weights().astype(np.float64)
    # two steps of (at most) lr each; coordinates whose gradient is at the
    # FP32 noise level may take the other sign
    big = (np.abs(g) > 1e-3 * np.abs(g).max()) & (np.abs(g2) > 1e-3 * np.abs(g2).max())
    assert big.mean() > 0.5
    assert np.abs(got - w2)[big].max() < 2e-5
    assert np.abs(got - w2).max() <= 1e-2
    h.close()


# ---------------------------------------------------------------------------
# The step with the network closure.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_rejected_network_falls_back_everywhere(precision):
    # a bound no proposal meets: every node takes the exact solve and the
    # step equals the exact one
    M = 3
    wl = W.random_mixture(M=M, shape=(5, 6, 7), seed=21, velocity=0.03)
    prm = oracle_params(wl)
    pops = O.init_populations(wl.X, wl.u, wl.T, wl.P, prm) * W.perturbation((M + 2, 27) + wl.shape, 0.01, 3)
    ha = gpu_handle(wl, precision)
    hb = gpu_handle(wl, precision, closure="mlp", closure_bound=1e-30)
    ha.set_populations(pops)
    hb.set_populations(pops)
    ha.step(2)
    hb.step(2)
    a, b = ha.populations(), hb.populations()
    assert rel(b, a) < 1e-6
    acc, fb = hb.closure_stats()
    assert acc == 0 and fb == 2 * wl.nodes
    ha.close()
    hb.close()


def _train_on_method(M, seed=31, shape=(16, 16, 16), amplitude=0.5, velocity=0.02):
    """Training pairs the method generates for one mixture (its constants from
    `seed`): exact-closure runs from a few initial fields, sampled at a few
    times, shuffled."""
    import torch
    feats, tgts = [], []
    for k in range(3):
        wl = W.random_mixture(M=M, shape=shape, seed=seed, field_seed=1000 + k, velocity=velocity,
                              amplitude=amplitude)
        h = gpu_handle(wl, "fp32")
        h.init_fields(wl.X, wl.u, wl.T, wl.P)
        for t in range(3):
            h.step(20)
            f, g = h.closure_samples()
            feats.append(f)
            tgts.append(g)
        h.close()
    feat = torch.cat(feats)
    tgt = torch.cat(tgts)
    perm = torch.randperm(feat.shape[0], generator=torch.Generator().manual_seed(seed)).to(feat.device)
    return feat[perm].contiguous(), tgt[perm].contiguous()


def test_trained_network_is_accepted_and_within_contract():
    """What the trained network gains: it replaces the exact solve at nearly
    every node (the fallback catches the rest) with every field within 1e-3
    of the FP64 oracle (FP32 storage), on a resting mixture whose composition
    varies by 10 %; on BF16 storage its error against the oracle stays at the
    storage's own (BF16 reaches ~2e-3 on the velocity of such states, see the
    reduced-precision parity tests; the chosen form's 1e-3 contract against
    the oracle is checked on the acoustic workload in test_gpu_parity.py)."""
    M = 3
    feat, tgt = _train_on_method(M, seed=31, amplitude=0.1, velocity=0.0)
    wl = W.random_mixture(M=M, shape=(8, 8, 8), seed=31, field_seed=77, amplitude=0.1)
    h = gpu_handle(wl, "fp32", closure="mlp")
    h.set_closure_weights(W.closure_initial_weights(M, seed=1))
    loss0, _ = h.closure_loss_grad(feat[:4096], tgt[:4096])
    h.closure_train(feat, tgt, batch=2048, steps=3000, lr=1e-3)
    last = h.closure_train(feat, tgt, batch=2048, steps=1000, lr=2e-4)
    assert last < 1e-2 * loss0
    w = h.closure_weights()
    prm = oracle_params(wl)
    nsteps = 20
    ref = O.run(O.init_populations(wl.X, wl.u, wl.T, wl.P, prm), prm, nsteps)
    mac = O.macroscopic(ref, prm)
    om = dict(rho=mac["rho"], u=mac["u"], T=mac["T"], P=mac["P"], X=mac["X"])
    mbar = float(np.dot(wl.X.reshape(M, -1).mean(axis=1), wl.molar_mass))
    cs = np.sqrt(1.4 * wl.T.mean() / mbar)
    h.init_fields(wl.X, wl.u, wl.T, wl.P)
    h.step(nsteps)
    acc, fb = h.closure_stats()
    assert acc + fb == nsteps * wl.nodes
    assert acc > 0.9 * (acc + fb), (acc, fb)
    errs = field_errors(h.moments_dict(), om, cs)
    assert max(errs.values()) < 1e-3, errs
    h.close()
    # BF16 storage: the network costs no accuracy beyond the storage's own
    errs = {}
    for closure in ("mlp", "exact"):
        hb = gpu_handle(wl, "bf16", closure=closure)
        if closure == "mlp":
            hb.set_closure_weights(w)
        hb.init_fields(wl.X, wl.u, wl.T, wl.P)
        hb.step(nsteps)
        errs[closure] = field_errors(hb.moments_dict(), om, cs)
        hb.close()
    for k in errs["exact"]:
        assert errs["mlp"][k] <= 1.5 * errs["exact"][k] + 2e-4, (k, errs)
