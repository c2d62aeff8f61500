"""The z-slab exchange schedule (paper_2004_11286_gb300.slabs.halo_exchange)
on world_size-2 gloo ranks, CPU only.  Each rank steps its slab of a small
grid with the FP64 oracle (periodic within the slab's extended planes, as the
CUDA handles are) and refreshes its three ghost planes on each side through
the schedule after every step, the buffers travelling by point-to-point
send / receive.  The interiors must equal the same planes of the undivided
oracle run: the schedule pairs the right faces and ranks, and three planes
cover what one step reads (collision neighbours, the two derivatives of the
non-local term of Eq. Xalpha, streaming)."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, walls, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    import oracle as O
    from paper_2004_11286_gb300 import workloads as W
    from paper_2004_11286_gb300.slabs import GHOST, extended_planes, halo_exchange, slab_bounds
    from gpu_helpers import oracle_params
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        shape = (12, 5, 6)
        wl = W.random_mixture(M=2, shape=shape, seed=77, velocity=0.02)
        prm = oracle_params(wl, walls_x=walls)
        full = O.init_populations(wl.X, wl.u, wl.T, wl.P, prm) * W.perturbation((4, 27) + shape, 0.005, 5)
        nz, g = shape[0], GHOST
        z0, z1 = slab_bounds(nz, world)[rank]
        mine = np.ascontiguousarray(full[:, :, extended_planes(z0, z1, g, nz)])
        ext = mine.shape[2]
        inbox = {}

        def pack(face):
            planes = slice(g, 2 * g) if face == 0 else slice(ext - 2 * g, ext - g)
            return torch.from_numpy(np.ascontiguousarray(mine[:, :, planes]))

        def unpack(face, buf):
            planes = slice(0, g) if face == 0 else slice(ext - g, ext)
            mine[:, :, planes] = buf.numpy()

        def transport(sends, recvs):
            ops = [dist.P2POp(dist.isend, buf, dst) for buf, dst in sends]
            bufs = [torch.empty_like(sends[0][0]) for _ in recvs]
            ops += [dist.P2POp(dist.irecv, b, src) for b, (face, src) in zip(bufs, recvs)]
            for r in dist.batch_isend_irecv(ops):
                r.wait()
            return bufs

        steps = 12
        for _ in range(steps):
            mine = O.step(mine, prm)
            halo_exchange(rank, world, pack, unpack, transport)
        ref = O.run(full, prm, steps)
        out.put((rank, float(np.abs(mine[:, :, g:ext - g] - ref[:, :, z0:z1]).max()),
                 bool(np.array_equal(mine[:, :, g:ext - g], ref[:, :, z0:z1]))))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("walls", [False, True])
def test_two_gloo_ranks_reproduce_the_undivided_grid(walls):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, walls, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, err, exact in sorted(res):
        assert err <= 1e-15 * 1.0, (rank, err)
        assert exact, (rank, err)
