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


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    from paper_2004_11286_gb300 import binding
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.LbmError) as e:
        binding.conserved_sums_noalloc(dummy, 8, (256, 256, 256), out)
    assert e.value.status == 1 and "static scratch" in str(e.value)
