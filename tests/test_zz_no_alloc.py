"""The allocation-free conservation sums (lbm_mix_conserved_sums_noalloc) agree
with lbm_mix_diagnostics.

The entry point exists for callers that cannot call cudaMalloc where they need
the sums (device memory owned by a pool or arena, plugins given only device
pointers, loops that must not allocate or synchronise); its scratch is a
static device array inside the library.  This file is collected last so that
a run stopping at the first failure has already run every other test.
"""

import numpy as np
import pytest

import oracle as O
from paper_2004_11286_gb300 import workloads as W

from gpu_helpers import gpu_handle, oracle_params

pytestmark = pytest.mark.gpu


def test_noalloc_sums_match_diagnostics_on_two_calls():
    import torch
    from paper_2004_11286_gb300 import binding, build
    build.build()
    wl = W.random_mixture(M=3, shape=(9, 10, 11), seed=5, velocity=0.02)
    prm = oracle_params(wl)
    pops = O.init_populations(wl.X, wl.u, wl.T, wl.P, prm) * W.perturbation((5, 27) + wl.shape, 0.01, 2)
    h = gpu_handle(wl, "fp64")
    h.set_populations(pops)
    dev = h.pops_buf.device
    dpops = torch.empty(pops.size, dtype=torch.float64, device=dev)
    sums = torch.full((wl.M + 5,), float("nan"), dtype=torch.float64, device=dev)
    for call in range(2):                      # two calls in a row on different states
        ref = h.diagnostics()
        h.populations(out=dpops)
        binding.conserved_sums_noalloc(dpops, wl.M, wl.shape, sums)
        got = sums.cpu().numpy()
        scale = np.maximum(np.abs(ref), np.abs(ref[wl.M]))
        assert np.all(np.abs(got - ref) <= 1e-12 * scale), (call, got, ref)
        h.step(3)
    h.close()


@pytest.mark.parametrize("M,shape", [
    (8, (48, 48, 48)),        # 432 blocks of partials: the final sum's strided loop over blocks
    (1, (257, 85, 512)),      # 11,184,640 nodes: exactly the scratch's capacity at M = 1
])
def test_noalloc_sums_at_many_blocks_and_at_the_cap(M, shape):
    """Against lbm_mix_diagnostics at 1e-12 on two states: more partial blocks
    than the final kernel's 256 threads (M = 8, the widest value set), and a
    grid of exactly (2^18 / (M + 5)) * 256 nodes, the largest the static
    scratch takes, next to one node more, which is refused."""
    import torch
    from paper_2004_11286_gb300 import binding, build
    build.build()
    wl = W.random_mixture(M=M, shape=shape, seed=11, modes=4)
    h = gpu_handle(wl, "fp64")
    h.init_fields(wl.X, wl.u, wl.T, wl.P)
    N = wl.nodes
    dev = h.pops_buf.device
    dpops = torch.empty((M + 2) * 27 * N, dtype=torch.float64, device=dev)
    sums = torch.full((M + 5,), float("nan"), dtype=torch.float64, device=dev)
    for call in range(2):
        h.step(1)
        ref = h.diagnostics()
        h.populations(out=dpops)
        binding.conserved_sums_noalloc(dpops, M, shape, sums)
        got = sums.cpu().numpy()
        scale = np.maximum(np.abs(ref), np.abs(ref[M]))
        assert np.all(np.abs(got - ref) <= 1e-12 * scale), (call, got, ref)
    if shape == (257, 85, 512):
        with pytest.raises(binding.LbmError):
            binding.conserved_sums_noalloc(dpops, M, (257, 85, 513), sums)
    h.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    from paper_2004_11286_gb300 import binding
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.LbmError) as e:
        binding.conserved_sums_noalloc(dummy, 8, (256, 256, 256), out)
    assert e.value.status == 1 and "static scratch" in str(e.value)
