"""z-slab decomposition of the step: slabs, their ghost planes and the halo
exchange between them.

A global grid of nz planes is cut along z into slabs of balanced plane
counts.  Each slab is a handle (``binding.LbmMix``) on its own planes plus
``ghost`` planes below and above, periodic in z within itself; every handle
shares one reference rest state (``LbmMix.set_reference``).  After every
step each ghost region is refreshed from the neighbouring slab's boundary
planes (``LbmMix.halo_pack`` / ``halo_unpack``: population slots, side fields,
equilibrium records).  One step reads across at most three planes, so with
ghost = 3 each slab's interior evolves exactly as the same planes of the
undivided grid.

The exchange schedule is ``halo_exchange``: slab k sends its top interior
planes (face 1) to slab k+1, whose bottom ghost region (face 0) receives
them, and its bottom interior planes (face 0) to slab k-1's top ghost region
(face 1); slab indices are periodic.  It is written once, over three
callables (pack, unpack, transport), and used by

  * ``SlabSet``: all slabs in one process (one GPU or several), buffers
    moved by device copies;
  * ``DistributedSlab``: one slab per rank of torch.distributed (NCCL on GPUs),
    buffers moved by point-to-point send / receive.
"""

from __future__ import annotations

from typing import Callable, List, Sequence, Tuple

import numpy as np

GHOST = 3


def slab_bounds(nz: int, nslabs: int) -> List[Tuple[int, int]]:
    """Interior plane ranges [z0, z1) of `nslabs` balanced slabs of nz planes."""
    if nslabs < 1 or nslabs > nz:
        raise ValueError("need 1 <= nslabs <= nz")
    edges = [(k * nz) // nslabs for k in range(nslabs + 1)]
    return [(edges[k], edges[k + 1]) for k in range(nslabs)]


def extended_planes(z0: int, z1: int, ghost: int, nz: int) -> np.ndarray:
    """Global plane indices (periodic) of a slab's planes, ghosts included."""
    return np.arange(z0 - ghost, z1 + ghost) % nz


def halo_exchange(rank: int, world: int, pack: Callable[[int], object], unpack: Callable[[int, object], None],
                  transport: Callable[[Sequence[Tuple[object, int]], Sequence[Tuple[int, int]]], List[object]]):
    """One refresh of slab `rank`'s ghost regions among `world` slabs.

    pack(face) returns that face's interior-plane buffer; unpack(face, buf)
    writes a received buffer into the face's ghost planes; transport(sends,
    recvs) delivers sends = [(buffer, destination)] and returns the buffers
    for recvs = [(face, source)] in order.  Face 1 goes up (to rank + 1, into
    its face 0), face 0 goes down (to rank - 1, into its face 1)."""
    up, down = (rank + 1) % world, (rank - 1) % world
    sends = [(pack(1), up), (pack(0), down)]
    recvs = [(0, down), (1, up)]
    bufs = transport(sends, recvs)
    for (face, _), buf in zip(recvs, bufs):
        unpack(face, buf)


def reference_state(wl_X, wl_T, wl_P, molar_mass, R_U: float = 1.0):
    """The reference rest state the library derives from whole fields (mean
    mole fractions, temperature and pressure), for slabs that must share it:
    mass fractions, temperature, density."""
    M = len(molar_mass)
    Xm = np.asarray(wl_X).reshape(M, -1).mean(axis=1)
    Xm = Xm / Xm.sum()
    mbar = float(np.dot(Xm, molar_mass))
    T = float(np.mean(wl_T))
    P = float(np.mean(wl_P))
    Y = Xm * np.asarray(molar_mass) / mbar
    return Y, T, P * mbar / (R_U * T)


class SlabSet:
    """All slabs of a z-decomposed grid in this process.

    ``make_handle(shape, device)`` creates a ``binding.LbmMix`` for a slab's
    extended grid; ``devices`` places slab k on devices[k % len(devices)]."""

    def __init__(self, make_handle, shape, nslabs: int, molar_mass, cv_molar, R_U: float = 1.0,
                 ghost: int = GHOST, devices=None, slaved: int = -1, weak: bool = False):
        import torch
        self._torch = torch
        self.shape = tuple(int(v) for v in shape)
        nz, ny, nx = self.shape
        self.ghost = int(ghost)
        self.bounds = slab_bounds(nz, nslabs)
        if min(z1 - z0 for z0, z1 in self.bounds) < self.ghost:
            raise ValueError("every slab needs at least `ghost` planes")
        self.molar_mass = np.asarray(molar_mass, dtype=np.float64)
        self.cv_molar = np.asarray(cv_molar, dtype=np.float64)
        self.R_U = float(R_U)
        self.slaved = int(slaved) if slaved >= 0 else len(self.molar_mass) - 1
        self.weak = bool(weak)
        devs = devices or [torch.device("cuda", torch.cuda.current_device())]
        self.handles = []
        for k, (z0, z1) in enumerate(self.bounds):
            dev = torch.device(devs[k % len(devs)])
            self.handles.append(make_handle((z1 - z0 + 2 * self.ghost, ny, nx), dev))
        self.M = self.handles[0].M
        self.bufs = [[torch.empty(h.halo_bytes(self.ghost), dtype=torch.uint8, device=h.device) for _ in range(2)]
                     for h in self.handles]

    def _slice(self, a, k):
        z0, z1 = self.bounds[k]
        idx = extended_planes(z0, z1, self.ghost, self.shape[0])
        return np.ascontiguousarray(np.asarray(a)[..., idx, :, :])

    def init_fields(self, X, u, T, P):
        Y, Tr, rho = reference_state(X, T, P, self.molar_mass, self.R_U)
        for k, h in enumerate(self.handles):
            h.set_reference(Y, Tr, rho)
            h.init_fields(self._slice(X, k), self._slice(u, k), self._slice(T, k), self._slice(P, k))

    def set_populations(self, pops):
        """Natural-layout full populations of the whole grid [S][27][nz][ny][nx]."""
        Y, Tr, rho = self._reference_from_pops(pops)
        for k, h in enumerate(self.handles):
            h.set_reference(Y, Tr, rho)
            h.set_populations(self._slice(pops, k))

    def _reference_from_pops(self, pops):
        """The reference the library derives from whole-grid populations: the
        mean zeroth moments (the slaved species taking the deficit under
        strong coupling), their mass fractions and temperature."""
        M = self.M
        z = np.asarray(pops).reshape(M + 2, 27, -1).sum(axis=1).mean(axis=1)
        r, rho, rhoE = z[:M].copy(), float(z[M]), float(z[M + 1])
        if not self.weak:
            others = sum(r[a] for a in range(M) if a != self.slaved)
            if rho - others > 0.0:
                r[self.slaved] = rho - others
        Y = r / r.sum()
        Cv = float(np.dot(Y, self.cv_molar * self.R_U / self.molar_mass))
        return Y, rhoE / (rho * Cv), rho

    def exchange(self):
        torch = self._torch
        K = len(self.handles)
        packed = [[None, None] for _ in range(K)]
        for k, h in enumerate(self.handles):
            h.halo_pack(1, self.ghost, self.bufs[k][1])
            h.halo_pack(0, self.ghost, self.bufs[k][0])
        for k in range(K):
            for f in (0, 1):
                packed[k][f] = self.bufs[k][f]
        # every pack is complete before the unpacks that read it
        for h in self.handles:
            h.stream.synchronize()

        for k, h in enumerate(self.handles):
            def pack(face, k=k):
                return packed[k][face]

            def unpack(face, buf, h=h):
                h.halo_unpack(face, self.ghost, buf.to(h.device) if buf.device != h.device else buf)

            def transport(sends, recvs, k=k):
                # the buffer slab k receives on face 0 is slab k-1's face 1, on face 1 slab k+1's face 0
                return [packed[src][1 - face] for face, src in recvs]

            halo_exchange(k, K, pack, unpack, transport)
        for h in self.handles:
            h.stream.synchronize()

    def step(self, n: int = 1):
        for _ in range(int(n)):
            for h in self.handles:
                h.step(1)
            self.exchange()

    def _interior(self, arr, k):
        g = self.ghost
        return arr[..., g:arr.shape[-3] - g, :, :]

    def populations(self):
        return np.concatenate([self._interior(h.populations(), k) for k, h in enumerate(self.handles)], axis=-3)

    def moments_dict(self):
        parts = [h.moments_dict() for h in self.handles]
        out = {}
        for key in parts[0]:
            out[key] = np.concatenate([self._interior(p[key], k) for k, p in enumerate(parts)], axis=-3)
        return out

    def close(self):
        for h in self.handles:
            h.close()


class DistributedSlab:
    """This rank's slab of a z-decomposed grid (one slab per rank of the
    default torch.distributed group, one GPU per rank).  The exchange sends
    the packed faces to the neighbouring ranks point to point."""

    def __init__(self, make_handle, shape, molar_mass, R_U: float = 1.0, ghost: int = GHOST, device=None):
        import torch
        import torch.distributed as dist
        self._torch, self._dist = torch, dist
        self.rank, self.world = dist.get_rank(), dist.get_world_size()
        self.shape = tuple(int(v) for v in shape)
        nz, ny, nx = self.shape
        self.ghost = int(ghost)
        self.bounds = slab_bounds(nz, self.world)
        z0, z1 = self.bounds[self.rank]
        if z1 - z0 < self.ghost:
            raise ValueError("every slab needs at least `ghost` planes")
        self.molar_mass = np.asarray(molar_mass, dtype=np.float64)
        self.R_U = float(R_U)
        self.h = make_handle((z1 - z0 + 2 * self.ghost, ny, nx), device)
        nb = self.h.halo_bytes(self.ghost)
        self.out = [torch.empty(nb, dtype=torch.uint8, device=self.h.device) for _ in range(2)]
        self.inb = [torch.empty(nb, dtype=torch.uint8, device=self.h.device) for _ in range(2)]

    def init_fields(self, X, u, T, P):
        """Whole-grid fields (every rank passes the same arrays)."""
        Y, Tr, rho = reference_state(X, T, P, self.molar_mass, self.R_U)
        z0, z1 = self.bounds[self.rank]
        idx = extended_planes(z0, z1, self.ghost, self.shape[0])
        sl = lambda a: np.ascontiguousarray(np.asarray(a)[..., idx, :, :])
        self.h.set_reference(Y, Tr, rho)
        self.h.init_fields(sl(X), sl(u), sl(T), sl(P))

    def init_local(self, X, u, T, P, reference):
        """This slab's own fields on its extended planes (ghosts included) and
        the reference state (Y, T, rho) every rank uses."""
        Y, Tr, rho = reference
        self.h.set_reference(Y, Tr, rho)
        self.h.init_fields(X, u, T, P)

    def exchange(self):
        dist = self._dist

        def pack(face):
            self.h.halo_pack(face, self.ghost, self.out[face])
            return self.out[face]

        def unpack(face, buf):
            self.h.halo_unpack(face, self.ghost, buf)

        def transport(sends, recvs):
            if self.world == 1:
                # the bottom ghosts take this slab's own top planes (sends[0]), the top ghosts its bottom ones
                return [sends[face][0] for face, _ in recvs]
            self.h.stream.synchronize()
            ops = [dist.P2POp(dist.isend, buf, dst) for buf, dst in sends]
            ops += [dist.P2POp(dist.irecv, self.inb[face], src) for face, src in recvs]
            for r in dist.batch_isend_irecv(ops):
                r.wait()
            return [self.inb[face] for face, _ in recvs]

        halo_exchange(self.rank, self.world, pack, unpack, transport)

    def step(self, n: int = 1):
        for _ in range(int(n)):
            self.h.step(1)
            self.exchange()

    def close(self):
        self.h.close()
