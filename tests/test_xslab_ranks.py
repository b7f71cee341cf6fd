"""The x-slab decomposition of one large lattice among ranks, on CPU with the oracle as each
rank's step (two gloo ranks).  A site's update reads the populations of the sites within two
columns (streaming brings them from one column away, and the non-ideal force needs the densities
of the neighbouring columns, which are formed from what streams into those), so a rank that owns
columns [x0, x0 + w) steps a window with two halo columns on each side, keeps the w interior
columns, and before the next step swaps two boundary columns of all 18 populations with each
neighbour.  The noise counters are the global lattice's (x periodic, walls local to every slab).
After every step the gathered slabs equal the undivided lattice bit for bit."""
import os
import socket

import numpy as np
import torch
import torch.multiprocessing as mp

import oracle

LX, LZ, STEPS, HALO = 16, 8, 12, 2
PARAMS = dict(kT=1e-4, G=0.3, grad_c0=0.02, seed=21, lattice_id=3)


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = LX // world
    x0 = rank * w
    left, right = (rank - 1) % world, (rank + 1) % world
    o = oracle.OracleLattice(w + 2 * HALO, LZ, **PARAMS)
    o.set_site_map((x0 - HALO) % LX, LX)
    slabs = []
    for t in range(STEPS):
        o.step(1)
        f = o.populations()
        inner = np.ascontiguousarray(f[..., HALO:HALO + w])
        # my first columns are the left neighbour's right halo and my last ones the right
        # neighbour's left halo; tags keep the two messages apart when both neighbours coincide
        to_left = torch.from_numpy(np.ascontiguousarray(inner[..., :HALO]))
        to_right = torch.from_numpy(np.ascontiguousarray(inner[..., w - HALO:]))
        from_left = torch.empty_like(to_left)
        from_right = torch.empty_like(to_right)
        reqs = [dist.isend(to_left, left, tag=1), dist.isend(to_right, right, tag=2),
                dist.irecv(from_right, right, tag=1), dist.irecv(from_left, left, tag=2)]
        for r in reqs:
            r.wait()
        o.set_populations(np.concatenate([from_left.numpy(), inner, from_right.numpy()], axis=-1))
        slabs.append(inner.ravel().tolist())
    out[rank] = slabs
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_slabs_with_halo_exchange_equal_the_whole_lattice():
    oracle.build()
    world = 2
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = {r: [np.array(s).reshape(2, 9, LZ, LX // world) for s in out[r]] for r in range(world)}
    whole = oracle.OracleLattice(LX, LZ, **PARAMS)
    for t in range(STEPS):
        whole.step(1)
        got = np.concatenate([res[r][t] for r in range(world)], axis=-1)
        np.testing.assert_array_equal(got, whole.populations(), err_msg=f"step {t}")
