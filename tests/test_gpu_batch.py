"""The batched ensemble (one launch per kernel for many independent domains,
graph-replayed step pairs, autotuned launch shapes) against single-domain
handles and the FP64 oracle."""

import numpy as np
import pytest

import oracle as O
from paper_2004_11286_gb300 import workloads as W

from gpu_helpers import oracle_params, rel

pytestmark = pytest.mark.gpu

SHAPES = [(5, 6, 7), (4, 4, 9), (3, 8, 5), (6, 5, 4)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2004_11286_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()


def _domains(shapes, seed0=500):
    return [W.ensemble_domain(s, seed0 + k) for k, s in enumerate(shapes)]


def _batch(wls, precision):
    from paper_2004_11286_gb300 import binding
    kws = [binding.workload_params(wl, precision=precision, slaved=W.slaved_species(wl)) for wl in wls]
    return binding.LbmBatch(kws)


def _perturbed(wl, prm, seed):
    pops = O.init_populations(wl.X, wl.u, wl.T, wl.P, prm)
    return pops * W.perturbation(pops.shape, 0.01, seed)


@pytest.mark.parametrize("precision,mode", [("fp32", 0), ("bf16", 0), ("bf16", 1)])
def test_batch_matches_single_domains(precision, mode):
    from gpu_helpers import gpu_handle
    wls = _domains(SHAPES)
    b = _batch(wls, precision)
    b.set_mode(mode, branches=3)
    singles = []
    for d, wl in enumerate(wls):
        prm = oracle_params(wl)
        pops = _perturbed(wl, prm, d)
        b.domain(d).set_populations(pops)
        h = gpu_handle(wl, precision)
        h.set_populations(pops)
        singles.append(h)
    b.step(5)                       # two graph replays and one single step
    b.step(2)                       # starts at the odd parity
    b.synchronize()
    for d, h in enumerate(singles):
        h.step(7)
        assert rel(b.domain(d).populations(), h.populations()) < 1e-6, d
        h.close()
    b.close()


def test_batch_fp64_matches_oracle():
    wls = _domains(SHAPES[:3], seed0=600)
    b = _batch(wls, "fp64")
    refs = []
    for d, wl in enumerate(wls):
        prm = oracle_params(wl)
        pops = _perturbed(wl, prm, 10 + d)
        b.domain(d).set_populations(pops)
        refs.append((prm, pops))
    b.step(3)
    for d, (prm, pops) in enumerate(refs):
        ref = O.run(pops, prm, 3)
        assert rel(b.domain(d).populations(), ref) < 1e-12, d
    b.close()


def test_autotune_restores_state_and_keeps_results():
    wls = _domains(SHAPES, seed0=700)
    b = _batch(wls, "bf16")
    for d, wl in enumerate(wls):
        b.domain(d).init_fields(wl.X, wl.u, wl.T, wl.P)
    before = [b.domain(d).populations().copy() for d in range(len(wls))]
    cfg = b.autotune(trial_steps=2)
    c = b.config()
    assert c["grid_collide"] == cfg["grid_collide"] and c["block_stencil"] in (128, 256)
    assert c["mode"] == cfg["mode"] in (0, 1) and c["branches"] == cfg["branches"]
    assert cfg["ms_per_step"] > 0
    for d in range(len(wls)):
        assert np.array_equal(b.domain(d).populations(), before[d])
        assert b.domain(d).step_count == 0
    b.step(4)
    tuned = [b.domain(d).populations().copy() for d in range(len(wls))]
    # the same steps with the default shapes (one block per tile) and no graphs
    b2 = _batch(wls, "bf16")
    for d, wl in enumerate(wls):
        b2.domain(d).init_fields(wl.X, wl.u, wl.T, wl.P)
    c2 = b2.config()
    b2.set_mode(0)
    b2.set_config(c2["tiles_collide"], 256, c2["tiles_256"], use_graph=False)
    b2.step(4)
    for d in range(len(wls)):
        assert rel(b2.domain(d).populations(), tuned[d]) < 1e-6
    b.close()
    b2.close()


def test_domain_stepped_alone_is_rejected():
    from paper_2004_11286_gb300 import binding
    wls = _domains(SHAPES[:2], seed0=800)
    b = _batch(wls, "fp32")
    for d, wl in enumerate(wls):
        b.domain(d).init_fields(wl.X, wl.u, wl.T, wl.P)
    b.domain(1).step(1)
    with pytest.raises(binding.LbmError) as e:
        b.step(1)
    assert e.value.status == 6
    b.close()
