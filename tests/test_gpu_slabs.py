"""z-slab decomposition on one GPU: two and three slab handles, each with
three ghost planes per side refreshed by halo pack / unpack after every
step, against one handle on the undivided grid sharing the same reference
state.  Every slab computes each of its interior nodes with the same
arithmetic on the same inputs, so the interiors must agree bit for bit:
FP64 and FP32, 16-bit storage (whose equilibrium records travel in the
halo), both AA parities over 100 steps, and the closed tube's x walls."""

import numpy as np
import pytest

from paper_2004_11286_gb300 import workloads as W
from paper_2004_11286_gb300.slabs import SlabSet, reference_state

from gpu_helpers import gpu_handle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2004_11286_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()


@pytest.mark.parametrize("precision,nslabs,walls,M", [
    ("fp64", 2, False, 3), ("fp64", 3, True, 3), ("fp32", 2, False, 2), ("fp32", 3, False, 8),
    ("bf16", 2, False, 3), ("fp16", 3, True, 2),
])
def test_slabs_reproduce_the_undivided_grid(precision, nslabs, walls, M):
    wl = W.random_mixture(M=M, shape=(12, 6, 8), seed=60 + M, velocity=0.02)
    Y, T, rho = reference_state(wl.X, wl.T, wl.P, wl.molar_mass, wl.R_U)
    one = gpu_handle(wl, precision, walls_x=walls)
    one.set_reference(Y, T, rho)
    one.init_fields(wl.X, wl.u, wl.T, wl.P)
    from paper_2004_11286_gb300 import binding

    def make(shape, dev):
        return binding.LbmMix(wl.molar_mass, wl.cv_molar, wl.D, mu=wl.mu, lam=wl.lam, shape=shape,
                              precision=precision, slaved=W.slaved_species(wl), R_U=wl.R_U, walls_x=walls,
                              device=dev)

    slabs = SlabSet(make, wl.shape, nslabs, wl.molar_mass, wl.cv_molar, wl.R_U, slaved=W.slaved_species(wl))
    slabs.init_fields(wl.X, wl.u, wl.T, wl.P)
    for chunk in (1, 1, 98):                   # parities 0, 1, then many
        one.step(chunk)
        slabs.step(chunk)
        a, b = slabs.populations(), one.populations()
        assert np.array_equal(a, b), (chunk, float(np.abs(a - b).max()))
    ma, mb = slabs.moments_dict(), one.moments_dict()
    for k in ("rho", "u", "T", "P", "X"):
        assert np.array_equal(ma[k], mb[k]), k
    one.close()
    slabs.close()


def test_halo_arguments_are_checked():
    from paper_2004_11286_gb300.binding import LbmError
    import torch
    wl = W.random_mixture(M=2, shape=(8, 4, 4), seed=1)
    h = gpu_handle(wl, "fp32")
    h.init_fields(wl.X, wl.u, wl.T, wl.P)
    buf = torch.empty(h.halo_bytes(2), dtype=torch.uint8, device=h.device)
    with pytest.raises(LbmError):
        h.halo_pack(2, 2, buf)                  # no such face
    with pytest.raises(LbmError):
        h.halo_pack(0, 3, buf)                  # nz = 8 < 3 * ghost
    h.halo_pack(0, 2, buf)
    h.halo_unpack(1, 2, buf)
    h.close()


def test_distributed_slab_on_one_rank_wraps_onto_itself():
    """DistributedSlab with a world of one rank: its two faces exchange with
    each other (the periodic grid through its own ghost planes), which must
    again reproduce one handle on the whole grid bit for bit."""
    import os
    import torch.distributed as dist
    from paper_2004_11286_gb300 import binding
    from paper_2004_11286_gb300.slabs import GHOST, DistributedSlab, extended_planes
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    os.environ.setdefault("MASTER_PORT", "29517")
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        wl = W.random_mixture(M=3, shape=(10, 6, 8), seed=71, velocity=0.02)
        Y, T, rho = reference_state(wl.X, wl.T, wl.P, wl.molar_mass, wl.R_U)

        def make(shape, dev):
            return binding.LbmMix(wl.molar_mass, wl.cv_molar, wl.D, mu=wl.mu, lam=wl.lam, shape=shape,
                                  precision="fp32", slaved=W.slaved_species(wl), R_U=wl.R_U)

        sl = DistributedSlab(make, wl.shape, wl.molar_mass, wl.R_U)
        sl.init_fields(wl.X, wl.u, wl.T, wl.P)
        one = gpu_handle(wl, "fp32")
        one.set_reference(Y, T, rho)
        one.init_fields(wl.X, wl.u, wl.T, wl.P)
        sl.step(7)
        one.step(7)
        a = sl.h.populations()[:, :, GHOST:-GHOST]
        assert np.array_equal(a, one.populations())
        sl.close()
        one.close()
    finally:
        dist.destroy_process_group()
