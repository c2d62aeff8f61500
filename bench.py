#!/usr/bin/env python
"""Benchmark of the fused multicomponent D3Q27 stream-and-collide step.

Workload (N = 1 GPU, the default line): the two-component Kelvin-Helmholtz
shear layer on a 256^3 periodic grid, M = 2 species (molar masses 2, 28),
plain FP32, i.e. 2 species + f + g lattices, 108 populations per node; the
chosen form (BF16-stored populations, then BF16 plus the learned
Stefan-Maxwell closure) on the same workload; per-field errors against the
FP64 oracle on a reduced copy of the workload; secondary lines for the
eight-species 192^3 mixture (FP32, BF16, BF16 + closure) and the 64-domain
ensemble.  One bench step = one lattice time step of the whole grid (all
lattices).  The populations (7.2 GB) are larger than L2, so no flush is
needed between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 oracle
(the only other implementation of the method) on a bounded periodic sample of
the same workload on the host cores.  Under torchrun each rank runs an
independent replica (value = all ranks' lattice updates / max time).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS (species+f+g) and HBM-roofline fraction, plain FP32 vs chosen form"
UNIT = "MLUPS"
FALLBACK_HBM_GBS = 6800.0


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # The double shear layer is unstable in the method itself (its FP64 oracle
    # diverges too): the default run stays well inside its first 100 steps.
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--n", type=int, default=None,
                    help="grid edge (shear layer: 256, acoustic pulse: 128, mixture: 192 by default)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the secondary lines (eight-species mixture, ensemble) of the default run")
    ap.add_argument("--no-parity", action="store_true", help="skip the per-field errors against the oracle")
    ap.add_argument("--decompose", action="store_true",
                    help="under torchrun: one z slab of a (n*N) x n x n grid per rank, ghost planes exchanged "
                         "point to point (NCCL) after every step, instead of independent replicas")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", choices=["shear", "acoustic", "ensemble", "mixture"], default="shear",
                    help="shear: the 256^3 two-component shear layer (default line); acoustic: the 128^3 "
                         "binary pulse; ensemble: 64 uneven ternary domains in one batched launch (BF16); "
                         "mixture: M-species (default 8) random mixture on an n^3 grid (default 192), FP32 "
                         "against BF16 and BF16 + learned closure")
    ap.add_argument("--M", type=int, default=8, help="species of the mixture workload")
    ap.add_argument("--no-chosen-form", action="store_true",
                    help="skip the BF16-storage / learned-closure comparison on the same workload")
    ap.add_argument("--oracle-sample", nargs=3, metavar=("WORKLOAD", "EDGE", "STEPS"),
                    help=argparse.SUPPRESS)
    return ap.parse_args()


# ---------------------------------------------------------------------------
# Replicas over ranks (N > 1): every rank runs its own copy of the workload
# (the step does not shard without a halo exchange); the job's time is the
# slowest rank's and its throughput all ranks' lattice updates over it.
# ---------------------------------------------------------------------------
def _max_over_ranks(x: float, world: int, device) -> float:
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_mlups(world: int, nodes: int, steps: int, seconds: float) -> float:
    return world * nodes * steps / seconds / 1e6


# ---------------------------------------------------------------------------
# Oracle timing (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------
def _workload(name: str, n: int):
    """The bench workloads (input recipes only; workloads.py)."""
    from paper_2004_11286_gb300 import workloads as W
    if name == "shear":
        return W.shear_layer(n=n)
    if name == "acoustic":
        return W.acoustic_pulse(n=n, sigma=6.0 * n / 128.0)
    raise ValueError(name)


def _oracle_sample_worker(name: str, edge: int, steps: int, warmup: int = 1):
    import numpy as np
    import oracle as O
    from paper_2004_11286_gb300 import workloads as W
    wl = _workload(name, edge)
    prm = O.Params(wl.molar_mass, wl.cv_molar, wl.D, mu=wl.mu, lam=wl.lam, slaved=W.slaved_species(wl))
    pops = O.init_populations(wl.X, wl.u, wl.T, wl.P, prm)
    for _ in range(warmup):
        pops = O.step(pops, prm)
    t0 = time.perf_counter()
    for _ in range(steps):
        pops = O.step(pops, prm)
    dt = time.perf_counter() - t0
    assert np.isfinite(pops).all()
    return dict(nodes=wl.nodes, steps=steps, seconds=dt, mlups=wl.nodes * steps / dt / 1e6)


def _oracle_env():
    return dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
                CUDA_VISIBLE_DEVICES="")


def _run_oracle_subprocess(name: str, edge: int, steps: int, timeout: float = 900.0):
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", name, str(edge), str(steps)],
                       capture_output=True, text=True, env=_oracle_env(), timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def _run_oracle_parallel(name: str, edge: int, steps: int, procs: int, timeout: float = 900.0):
    """`procs` independent single-threaded oracle processes on the same
    sample at once (one per host core): whole-host throughput = all their
    lattice updates over the slowest one's time."""
    ps = [subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-sample", name, str(edge), str(steps)],
                           stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=_oracle_env())
          for _ in range(procs)]
    res = []
    for p in ps:
        out, err = p.communicate(timeout=timeout)
        if p.returncode != 0:
            raise RuntimeError("oracle sample failed: " + err[-2000:])
        res.append(json.loads(out.strip().splitlines()[-1]))
    secs = max(r["seconds"] for r in res)
    ups = sum(r["nodes"] * r["steps"] for r in res)
    return dict(mlups=ups / secs / 1e6, seconds=secs, procs=procs, nodes=res[0]["nodes"], steps=steps)


def _cpu_baseline(name: str, target_seconds: float = 15.0):
    cal = _run_oracle_subprocess(name, 16, 2)
    per_node_step = cal["seconds"] / (cal["nodes"] * cal["steps"])
    edge = 32
    steps = max(2, int(target_seconds / (per_node_step * edge ** 3)))
    one = _run_oracle_subprocess(name, edge, steps)
    cores = os.cpu_count() or 1
    allc = _run_oracle_parallel(name, edge, steps, cores)
    return {"value": round(allc["mlups"], 5), "unit": UNIT, "cores": cores, "kind": "oracle",
            "one_core": round(one["mlups"], 5),
            "sample": f"{name} recipe on a {edge}^3 periodic grid, {steps} steps, FP64 NumPy oracle: "
                      f"{cores} single-threaded processes at once on the host's {cores} cores "
                      f"({allc['seconds']:.1f} s), and one alone ({one['seconds']:.1f} s, `one_core`)"}


# ---------------------------------------------------------------------------
# Clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.samples = []
        self.proc = None
        self.window = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.perf_counter(), [v.strip() for v in line.split(",")]))

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        t0, t1 = self.window if self.window else (0, float("inf"))
        inside = [s for (t, s) in self.samples if t0 - 0.15 <= t <= t1 + 0.15] or [s for (_, s) in self.samples]
        if not inside:
            return None
        sm = [float(s[1]) for s in inside if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in inside if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in inside for k in range(4) if len(s) > 5 + k and s[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside)}


def _physical_gpu_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    parts = [p for p in vis.split(",") if p.strip()]
    if parts and all(p.strip().isdigit() for p in parts) and local_rank < len(parts):
        return int(parts[local_rank])
    return local_rank


# ---------------------------------------------------------------------------
# Roofline bookkeeping
# ---------------------------------------------------------------------------
def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        for key in ("hbm_gbs", "hbm_GBps", "copy_gbs"):
            if key in d:
                return float(d[key]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def _kernel_source_hash():
    """Hash of the kernel sources and the compiler flags they are built with."""
    from paper_2004_11286_gb300 import build
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2004_11286_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    h.update(" ".join(build.NVCC_FLAGS).encode())
    return h.hexdigest()[:16]


def _recorded_traffic(kernel: str, precision: str, M: int, nodes: int, workload: str = "shear"):
    """DRAM bytes per launch from the committed ncu summary of this workload,
    if it was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get(f"{workload}/{kernel}/{precision}/M{M}")
    if not e or e.get("source_hash") != _kernel_source_hash():
        return None
    return float(e["bytes_per_node"]) * nodes


def _algorithmic_bytes(M: int, precision: str):
    """Per-node algorithmic bytes of each kernel and of the whole step."""
    b = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}[precision]
    bs = 8 if precision == "fp64" else 4
    S = M + 2
    # 16-bit storage: each node's equilibrium record (rec_w floats) written
    # once and read once (its receivers gather it from L1/L2)
    rec = 2 * 4 * (8 + ((1 + M + 3) // 4) * 4) if b == 2 else 0
    return {
        # every population read + written once; the senders' deferred terms
        # (X, K, theta) read once per node; this node's 7 side fields written
        "collide_stream": 2 * 27 * S * b + 7 * bs + 7 * bs + rec,
        "grad_GK": 7 * bs + 7 * bs,                 # Phi, c_omega, C_p, s, theta -> G, K, theta
        "grad_X": 3 * bs + 3 * bs,                  # G -> X
        "step": 2 * 27 * S * b + 2 * 5 * bs + rec,  # method minimum: populations once + side fields once
    }


# ---------------------------------------------------------------------------
# The chosen form on the same workload: BF16-stored populations, then BF16
# plus the learned Stefan-Maxwell closure (network trained here on pairs the
# exact method generates from this workload, exact fallback).
# ---------------------------------------------------------------------------
def _chosen_form(wl, dev, steps: int, peak: float):
    import torch
    from paper_2004_11286_gb300 import binding, workloads as W
    slaved = W.slaved_species(wl)
    N = wl.nodes
    out = {}

    def timed(h, k):
        h.init_fields(wl.X, wl.u, wl.T, wl.P)
        h.step(5)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(h.stream)
        h.step(k)
        e1.record(h.stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / k

    alg = _algorithmic_bytes(wl.M, "bf16")["step"]
    hb = binding.from_workload(wl, precision="bf16", slaved=slaved, device=dev)
    ms = timed(hb, steps)
    hb.close()
    out["bf16"] = {"MLUPS": round(N / ms / 1e3, 2), "ms_per_step": round(ms, 5),
                   "step_frac": round(alg * N / (ms * 1e-3) / 1e9 / peak, 4)}
    # training pairs from the exact method on this workload, then Adam
    t0 = time.perf_counter()
    hs = binding.from_workload(wl, precision="fp32", slaved=slaved, device=dev)
    hs.init_fields(wl.X, wl.u, wl.T, wl.P)
    feats, tgts = [], []
    for _ in range(3):
        hs.step(20)
        f, g = hs.closure_samples()
        idx = torch.randperm(N, generator=torch.Generator().manual_seed(len(feats)))[: min(N, 1 << 18)].to(dev)
        feats.append(f[idx])
        tgts.append(g[idx])
    hs.close()
    feat = torch.cat(feats).contiguous()
    tgt = torch.cat(tgts).contiguous()
    hm = binding.from_workload(wl, precision="bf16", slaved=slaved, closure="mlp", device=dev)
    hm.set_closure_weights(W.closure_initial_weights(wl.M, seed=1))
    loss = None
    for k, lr in ((3000, 1e-3), (1500, 2e-4)):
        loss = hm.closure_train(feat, tgt, batch=4096, steps=k, lr=lr)
    train_s = time.perf_counter() - t0
    hm.closure_stats(reset=True)
    ms = timed(hm, max(50, steps // 4))
    acc, fb = hm.closure_stats()
    hm.close()
    out["bf16_learned_closure"] = {
        "MLUPS": round(N / ms / 1e3, 2), "ms_per_step": round(ms, 5),
        "step_frac": round(alg * N / (ms * 1e-3) / 1e9 / peak, 4),
        "accepted_fraction": round(acc / max(1, acc + fb), 5), "residual_bound": 1e-2,
        "train": {"pairs": int(feat.shape[0]), "adam_steps": 4500, "last_loss": loss, "seconds": round(train_s, 2)}}
    return out


# ---------------------------------------------------------------------------
# Secondary workloads (not the default line): the batched ensemble and the
# eight-species mixture.
# ---------------------------------------------------------------------------
def _timed_steps(step, stream, k):
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def _bench_ensemble(a, dev):
    from paper_2004_11286_gb300 import binding, workloads as W
    shapes = W.ensemble_shapes(64, seed=4)
    kws, wls = [], []
    for k, sh in enumerate(shapes):
        wl = W.ensemble_domain(sh, 100 + k)
        kws.append(binding.workload_params(wl, precision="bf16", slaved=W.slaved_species(wl)))
    b = binding.LbmBatch(kws, device=dev)
    for k, sh in enumerate(shapes):
        wl = W.ensemble_domain(sh, 100 + k)
        b.domain(k).init_fields(wl.X, wl.u, wl.T, wl.P)
    cfg = b.autotune(trial_steps=3)
    b.step(a.warmup)
    b.synchronize()
    clocks = ClockSampler(_physical_gpu_index(0))
    time.sleep(0.3)
    t0 = time.perf_counter()
    ms = _timed_steps(b.step, b.stream, a.steps)
    clocks.mark(t0, time.perf_counter())
    b.synchronize()
    clk = clocks.stop()
    N = b.nodes
    value = N * a.steps / (ms * 1e-3) / 1e6
    peak, src = _peaks()
    alg = _algorithmic_bytes(3, "bf16")["step"]
    line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": 1, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": round(ms / a.steps, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "batched ensemble: 64 ternary diffusion domains, edges uniform in 32..96 "
                                   f"({N} nodes), M=3 (m=2,40,16), BF16 storage, FP32 arithmetic, one launch "
                                   "per kernel for all domains, step pairs as a CUDA graph",
                       "autotuned": cfg, "l2": "inputs larger than L2, no flush"},
            "roofline": {"bound": "hbm", "step_frac": round(alg * N * a.steps / (ms * 1e-3) / 1e9 / peak, 4),
                         "peak": peak, "unit": "GB/s", "step_algorithmic_bytes_per_node": alg},
            "clocks": clk}
    b.close()
    return line


def _bench_mixture(a, dev):
    import torch
    from paper_2004_11286_gb300 import binding, workloads as W
    M = a.M
    n = a.n if a.n is not None else 192
    wl = W.random_mixture(M=M, n=n, seed=7)
    slaved = W.slaved_species(wl)
    N = wl.nodes
    peak, src = _peaks()
    out = {}
    h = binding.from_workload(wl, precision="fp32", slaved=slaved, device=dev)
    h.init_fields(wl.X, wl.u, wl.T, wl.P)
    h.step(a.warmup)
    # 2^21 (2.1e6) training pairs the exact method generates from this
    # workload: 8 states 20 steps apart, 2^18 random nodes of each
    feats, tgts = [], []
    for _ in range(8):
        h.step(20)
        f, g = h.closure_samples()
        idx = torch.randperm(N, generator=torch.Generator().manual_seed(len(feats)))[: 1 << 18].to(dev)
        feats.append(f[idx].clone())
        tgts.append(g[idx].clone())
        del f, g
    ms = _timed_steps(h.step, h.stream, a.steps)
    h.close()
    alg32 = _algorithmic_bytes(M, "fp32")["step"]
    out["fp32"] = {"MLUPS": round(N * a.steps / ms / 1e3, 2), "ms_per_step": round(ms / a.steps, 4),
                   "step_frac": round(alg32 * N * a.steps / (ms * 1e-3) / 1e9 / peak, 4)}
    alg16 = _algorithmic_bytes(M, "bf16")["step"]
    hb = binding.from_workload(wl, precision="bf16", slaved=slaved, device=dev)
    hb.init_fields(wl.X, wl.u, wl.T, wl.P)
    hb.step(a.warmup)
    ms = _timed_steps(hb.step, hb.stream, a.steps)
    hb.close()
    out["bf16"] = {"MLUPS": round(N * a.steps / ms / 1e3, 2), "ms_per_step": round(ms / a.steps, 4),
                   "step_frac": round(alg16 * N * a.steps / (ms * 1e-3) / 1e9 / peak, 4)}
    feat = torch.cat(feats).contiguous()
    tgt = torch.cat(tgts).contiguous()
    hm = binding.from_workload(wl, precision="bf16", slaved=slaved, closure="mlp", device=dev)
    hm.set_closure_weights(W.closure_initial_weights(M, seed=1))
    t0 = time.perf_counter()
    for k, lr in ((4000, 1e-3), (2000, 2e-4)):
        loss = hm.closure_train(feat, tgt, batch=4096, steps=k, lr=lr)
    train_s = time.perf_counter() - t0
    hm.init_fields(wl.X, wl.u, wl.T, wl.P)
    hm.step(a.warmup)
    hm.closure_stats(reset=True)
    ms = _timed_steps(hm.step, hm.stream, a.steps)
    acc, fb = hm.closure_stats()
    hm.close()
    out["bf16_learned_closure"] = {"MLUPS": round(N * a.steps / ms / 1e3, 2), "ms_per_step": round(ms / a.steps, 4),
                                   "step_frac": round(alg16 * N * a.steps / (ms * 1e-3) / 1e9 / peak, 4),
                                   "accepted_fraction": round(acc / max(1, acc + fb), 5),
                                   "train": {"pairs": int(feat.shape[0]), "adam_steps": 6000, "last_loss": loss,
                                             "seconds": round(train_s, 2)}}
    line = {"metric": METRIC, "value": out["fp32"]["MLUPS"], "unit": UNIT, "n_gpus": 1, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": out["fp32"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"random {M}-species mixture, {n}^3 periodic, smooth 16-mode composition "
                                   "field, m_a in [2,44], D_ab log-uniform in [0.005, 0.1]"},
            "chosen_form": out}
    return line


# ---------------------------------------------------------------------------
def _bench_decomposed(a, name, dev, rank, world):
    """Weak scaling over a z-slab decomposition: the global grid is
    (n * world) x n x n; rank r steps its n planes plus three ghost planes
    per side and exchanges them with ranks r +- 1 after every step
    (slabs.DistributedSlab, NCCL point to point).  Each rank draws its own
    slab of the recipe (the shear layer varies along y only, so every slab
    has the same mean state and reference)."""
    import torch
    import torch.distributed as dist
    from paper_2004_11286_gb300 import binding, workloads as W
    from paper_2004_11286_gb300.slabs import GHOST, DistributedSlab, reference_state
    n = a.n
    ext = (n + 2 * GHOST, n, n)
    wl = W.shear_layer(shape=ext, seed=1234 + rank) if name == "shear" else W.acoustic_pulse(shape=ext)
    slaved = W.slaved_species(wl)

    def make(shape, device):
        return binding.LbmMix(wl.molar_mass, wl.cv_molar, wl.D, mu=wl.mu, lam=wl.lam, shape=shape,
                              precision=a.precision, slaved=slaved, R_U=wl.R_U, device=dev)

    sl = DistributedSlab(make, (n * world, n, n), wl.molar_mass, wl.R_U)
    sl.init_local(wl.X, wl.u, wl.T, wl.P, reference_state(wl.X, wl.T, wl.P, wl.molar_mass, wl.R_U))
    sl.step(a.warmup)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(_physical_gpu_index(int(os.environ.get("LOCAL_RANK", "0")))) if rank == 0 else None
    dist.barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(sl.h.stream)
    sl.step(a.steps)
    ev1.record(sl.h.stream)
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    dist.barrier()
    ms = _max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    clk = None
    if clocks is not None:
        clocks.mark(t0, t1)
        clk = clocks.stop()
    nodes = n ** 3
    sl.close()
    return {"metric": METRIC, "value": round(_job_mlups(world, nodes, a.steps, ms * 1e-3), 2), "unit": UNIT,
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(ms / a.steps, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if a.precision == "fp32" else a.precision, "data": "synthetic",
            "config": {"workload": f"{name} recipe, z-slab decomposition of a {n * world}x{n}x{n} grid, {n}^3 "
                                   f"interior planes per rank plus {GHOST} ghost planes per side exchanged by "
                                   "NCCL point-to-point after every step", "parallelism": f"z slabs x{world}",
                       "l2": "inputs larger than L2, no flush"},
            "clocks": clk, "gpu_launches": int(a.steps * 3 + a.steps * (6 if a.precision in ("fp16", "bf16") else 4))}


def _parity(name: str, dev):
    """Per-field errors against the FP64 oracle on a reduced copy of the
    workload (same recipe and constants, a grid the oracle steps in seconds),
    for plain FP32, BF16 storage and BF16 + the learned closure (trained on
    this copy's own exact pairs).  rho, T, P relative; u relative to
    max(||u||, 1e-3 c_s); X absolute (the norms of the parity tests)."""
    import numpy as np
    import torch
    import oracle as O
    from paper_2004_11286_gb300 import binding, workloads as W
    if name == "shear":
        wl, steps = W.shear_layer(shape=(16, 64, 16)), 20
    else:
        wl, steps = W.acoustic_pulse(shape=(12, 14, 16), sigma=2.0), 300
    slaved = W.slaved_species(wl)
    prm = O.Params(wl.molar_mass, wl.cv_molar, wl.D, mu=wl.mu, lam=wl.lam, slaved=slaved)
    mac = O.macroscopic(O.run(O.init_populations(wl.X, wl.u, wl.T, wl.P, prm), prm, steps), prm)
    mbar = float(np.dot(wl.X.reshape(wl.M, -1).mean(axis=1), wl.molar_mass))
    cs = float(np.sqrt(1.4 * wl.T.mean() / mbar))

    def errs(h):
        g = h.moments_dict()
        r = lambda k, fl=0.0: float(np.abs(g[k] - mac[k]).max() / max(float(np.abs(mac[k]).max()), fl))
        return {"rho": r("rho"), "u": r("u", 1e-3 * cs), "T": r("T"), "P": r("P"),
                "X": float(np.abs(g["X"] - mac["X"]).max())}

    out = {"workload": f"{name} recipe on {'x'.join(map(str, wl.shape))}, {steps} steps", "norm":
           "max|a-b| / max(|b|_inf, floor); floor 1e-3 c_s for u; X absolute"}
    for prec in ("fp32", "bf16"):
        h = binding.from_workload(wl, precision=prec, slaved=slaved, device=dev)
        h.init_fields(wl.X, wl.u, wl.T, wl.P)
        h.step(steps)
        out[prec] = {k: float(f"{v:.3g}") for k, v in errs(h).items()}
        h.close()
    hs = binding.from_workload(wl, precision="fp32", slaved=slaved, device=dev)
    hs.init_fields(wl.X, wl.u, wl.T, wl.P)
    feats, tgts = [], []
    for _ in range(4):
        hs.step(max(1, steps // 4))
        f, g = hs.closure_samples()
        feats.append(f)
        tgts.append(g)
    hs.close()
    feat, tgt = torch.cat(feats).contiguous(), torch.cat(tgts).contiguous()
    hm = binding.from_workload(wl, precision="bf16", slaved=slaved, closure="mlp", device=dev)
    hm.set_closure_weights(W.closure_initial_weights(wl.M, seed=1))
    hm.closure_train(feat, tgt, batch=2048, steps=2000, lr=1e-3)
    hm.closure_train(feat, tgt, batch=2048, steps=1000, lr=2e-4)
    hm.init_fields(wl.X, wl.u, wl.T, wl.P)
    hm.closure_stats(reset=True)
    hm.step(steps)
    acc, fb = hm.closure_stats()
    out["bf16_learned_closure"] = {k: float(f"{v:.3g}") for k, v in errs(hm).items()}
    out["bf16_learned_closure"]["accepted_fraction"] = round(acc / max(1, acc + fb), 4)
    hm.close()
    return out


def main():
    a = _args()
    if a.n is None:
        a.n = {"shear": 256, "acoustic": 128}.get(a.workload)
    if a.oracle_sample:
        name, edge, steps = a.oracle_sample
        print(json.dumps(_oracle_sample_worker(name, int(edge), int(steps))))
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    name = a.workload if a.workload in ("shear", "acoustic") else "shear"

    if a.impl == "reference":
        if rank != 0:
            return
        cal = _run_oracle_subprocess(name, 16, 2)
        per = cal["seconds"] / (cal["nodes"] * cal["steps"])
        budget = 120.0 / max(1, a.steps + a.warmup)
        # at most 48^3 per process, so one copy per core stays within the host's memory
        edge = int(max(8, min(a.n or 256, 48, round((budget / per) ** (1.0 / 3.0)))))
        cores = os.cpu_count() or 1
        res = _run_oracle_parallel(name, edge, a.steps, cores, timeout=1800)
        v = round(res["mlups"], 6)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
                "steps": a.steps, "warmup": a.warmup,
                "ms_per_step": round(1e3 * res["seconds"] / a.steps, 4), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"{name} recipe, {edge}^3 periodic sample of the {a.n}^3 workload, "
                                       f"{cores} single-threaded oracle processes", "precision": "fp64"},
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": f"{edge}^3 periodic grid, {a.steps} steps, one copy per core"},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import numpy as np
    import torch
    from paper_2004_11286_gb300 import binding, build, workloads as W

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    binding.load_library()
    if a.workload in ("ensemble", "mixture"):
        line = _bench_ensemble(a, dev) if a.workload == "ensemble" else _bench_mixture(a, dev)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return

    if world > 1 and a.decompose:
        line = _bench_decomposed(a, name, dev, rank, world)
        if rank == 0:
            print(json.dumps(line), flush=True)
        dist.destroy_process_group()
        return

    wl = _workload(name, a.n)
    slaved = W.slaved_species(wl)
    h = binding.LbmMix(wl.molar_mass, wl.cv_molar, wl.D, mu=wl.mu, lam=wl.lam, shape=wl.shape,
                       precision=a.precision, slaved=slaved, R_U=wl.R_U, device=dev)
    stream = h.stream
    Xd = torch.from_numpy(wl.X.ravel()).to(dev)
    ud = torch.from_numpy(wl.u.ravel()).to(dev)
    Td = torch.from_numpy(wl.T.ravel()).to(dev)
    Pd = torch.from_numpy(wl.P.ravel()).to(dev)
    h.init_fields(Xd, ud, Td, Pd)
    del Xd, ud, Td, Pd
    h.step(a.warmup)
    h.synchronize()

    # ---- device-timed region --------------------------------------------
    clocks = ClockSampler(_physical_gpu_index(local_rank))
    time.sleep(0.3)
    h.enable_kernel_timing(True)
    h.kernel_times()                                   # clear
    launches0 = h.launch_count
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t_host0 = time.perf_counter()
    ev0.record(stream)
    h.step(a.steps)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    t_host1 = time.perf_counter()
    if world > 1:
        dist.barrier()
    clocks.mark(t_host0, t_host1)
    launches = h.launch_count - launches0
    kt = h.kernel_times()
    h.enable_kernel_timing(False)
    h.synchronize()
    clk = clocks.stop()
    elapsed_ms = _max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    N = wl.nodes
    value = _job_mlups(world, N, a.steps, elapsed_ms * 1e-3)

    # ---- roofline of the dominant kernel ----------------------------------
    alg = _algorithmic_bytes(wl.M, a.precision)
    dom = max(kt, key=lambda k: kt[k][0])
    dom_ms = kt[dom][0] / max(1, kt[dom][1])
    peak, peak_src = _peaks()
    achieved = alg[dom] * N / (dom_ms * 1e-3) / 1e9
    step_alg_gbs = alg["step"] * N * a.steps / (elapsed_ms * 1e-3) / 1e9
    traffic = _recorded_traffic(dom, a.precision, wl.M, N, name)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": dom,
                "peak_source": peak_src + (" (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
                                           else " (6.8 TB/s, profiling recipe)"),
                "algorithmic_bytes_per_node": alg[dom],
                "kernel_ms_avg": round(dom_ms, 5),
                "kernel_share": {k: round(v[0] / max(1e-9, sum(x[0] for x in kt.values())), 4) for k, v in kt.items()},
                "step_algorithmic_bytes_per_node": alg["step"],
                "step_frac": round(step_alg_gbs / peak, 4)}

    # ---- end to end through the public API with host buffers ---------------
    e2e = None
    if not a.no_e2e:
        Xp = torch.from_numpy(wl.X.ravel()).pin_memory()
        up = torch.from_numpy(wl.u.ravel()).pin_memory()
        Tp = torch.from_numpy(wl.T.ravel()).pin_memory()
        Pp = torch.from_numpy(wl.P.ravel()).pin_memory()
        outp = torch.empty(h.n_outputs * N, dtype=torch.float64).pin_memory()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        h.init_fields(Xp, up, Tp, Pp)
        h.step(a.steps)
        h.moments(outp)
        sums = h.diagnostics()
        t1 = time.perf_counter()
        e2e_s = _max_over_ranks(t1 - t0, world, dev)
        assert np.isfinite(sums).all()
        h2d = (wl.M + 5) * N * 8
        d2h = h.n_outputs * N * 8 + (wl.M + 5) * 8
        e2e = {"value": round(_job_mlups(world, N, a.steps, e2e_s), 2), "unit": UNIT,
               "h2d_bytes_per_step": round(h2d / a.steps, 1), "d2h_bytes_per_step": round(d2h / a.steps, 1),
               "note": "init_fields from pinned host fields + step(K) + get_moments to pinned host + "
                       "diagnostics, host wall clock"}
        del Xp, up, Tp, Pp, outp
    h.close()
    torch.cuda.empty_cache()

    chosen = None
    if not a.no_chosen_form and a.precision == "fp32":
        chosen = _chosen_form(wl, dev, min(a.steps, 200), peak)

    parity = None
    if not a.no_parity and rank == 0:
        parity = _parity(name, dev)

    secondary = None
    if not a.no_secondary and world == 1 and rank == 0:
        torch.cuda.empty_cache()
        sa = argparse.Namespace(**vars(a))
        sa.steps, sa.warmup, sa.n, sa.M = min(a.steps, 60), 5, 192, 8
        secondary = {"mixture_M8_192cube": _bench_mixture(sa, dev)}
        torch.cuda.empty_cache()
        sa.steps = min(a.steps, 100)
        secondary["ensemble_64_domains"] = _bench_ensemble(sa, dev)
        for v in secondary.values():
            for k in ("metric", "unit", "n_gpus", "higher_is_better", "scaling", "vs_baseline", "data"):
                v.pop(k, None)

    cpu = None
    if rank == 0 and not a.no_cpu_baseline and world == 1:
        try:
            cpu = _cpu_baseline(name)
        except Exception as ex:  # the baseline is reported, never required
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"failed: {ex}"[:300]}

    if rank == 0:
        desc = {"shear": f"two-component Kelvin-Helmholtz shear layer, {a.n}^3 periodic D3Q27, M=2 (m=2,28), "
                         "tanh velocity and composition profiles, Mach 0.3",
                "acoustic": f"binary acoustic pulse, {a.n}^3 periodic D3Q27, M=2 (m=4,40)"}[name]
        line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": round(elapsed_ms / a.steps, 5), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if a.precision == "fp32" else a.precision,
                "data": "synthetic",
                "config": {"workload": f"{desc}, species+f+g = {27 * (wl.M + 2)} populations/node, {a.precision}",
                           "grid": list(wl.shape), "M": wl.M, "precision": a.precision,
                           "l2": "inputs larger than L2 (%.0f MB of populations), no flush" %
                                 (27 * (wl.M + 2) * N * {"fp64": 8, "fp32": 4}.get(a.precision, 2) / 1e6),
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "chosen_form": chosen, "parity": parity, "secondary": secondary,
                "gpu_launches": int(launches)}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
