"""The x-slab decomposition of one large lattice on the GPU (the library's site map and column
export/import): two processes, each stepping its slab as a window with two halo columns on each
side (its own context on the one GPU), swap two boundary columns of all 18 populations with each
neighbour after every step through host buffers over gloo.  The kernels of the two processes
never wait on each other: each step is a complete launch, and the exchange happens on the host
between steps.  After 12 steps the gathered slabs equal the undivided lattice run by the library
bit for bit, and the oracle within the parity bars (Sec. II.A: periodic in x, walls local to
every slab; the noise counters are the undivided lattice's)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1808_05168_gb300 import LatticeParams, Simulation, capi

pytestmark = pytest.mark.gpu

LX, LZ, STEPS, HALO = 512, 16, 12, 2
PARAMS = dict(lambda_s=1.1, lambda_d=0.9, kT=1e-4, G=0.3, grad_c0=0.02, seed=21, lattice_id=3)
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _worker(rank, world, port, prec, kw, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = LX // world
    x0 = rank * w
    left, right = (rank - 1) % world, (rank + 1) % world
    stream = torch.cuda.Stream()  # the library's kernels and torch's copies in one stream order
    with Simulation(LatticeParams(w + 2 * HALO, LZ, **PARAMS), precision=prec, **kw) as sim, \
            torch.cuda.stream(stream):
        sim.set_stream(stream)
        sim.set_site_map((x0 - HALO) % LX, LX)
        for _ in range(STEPS):
            sim.step(1)
            # my first owned columns are the left neighbour's right halo, my last ones the right
            # neighbour's left halo; tags keep the two messages apart when both are one process
            to_left = sim.export_columns(HALO, HALO).cpu()
            to_right = sim.export_columns(w, HALO).cpu()
            from_left, from_right = torch.empty_like(to_left), torch.empty_like(to_right)
            reqs = [dist.isend(to_left, left, tag=1), dist.isend(to_right, right, tag=2),
                    dist.irecv(from_right, right, tag=1), dist.irecv(from_left, left, tag=2)]
            for r in reqs:
                r.wait()
            sim.import_columns(0, from_left.cuda())
            sim.import_columns(w + HALO, from_right.cuda())
        out[rank] = np.ascontiguousarray(sim.populations()[..., HALO:HALO + w]).tobytes()
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("prec,kw", [("fp64", {}), ("dev32", {}), ("dev32", dict(graph=True, persistent=True))],
                         ids=["fp64", "dev32", "dev32-persistent"])
def test_two_gpu_slabs_with_halo_exchange_equal_the_whole_lattice(prec, kw):
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), prec, kw, out), nprocs=world, join=True)
        got = np.concatenate([np.frombuffer(out[r], np.float64).reshape(2, 9, LZ, LX // world)
                              for r in range(world)], axis=-1)
    with Simulation(LatticeParams(LX, LZ, **PARAMS), precision=prec, **kw) as sim:
        sim.step(STEPS)
        whole = sim.populations()
    np.testing.assert_array_equal(got, whole)
    o = oracle.OracleLattice(LX, LZ, omp=True, **PARAMS)
    o.step(STEPS)
    want = o.populations()
    if prec == "fp64":
        assert np.max(np.abs(got - want) / np.abs(want)) <= 1e-12
    else:
        z = np.arange(LZ) + 0.5 - LZ / 2
        c0 = 0.5 + z * PARAMS["grad_c0"]
        b = np.stack([W[:, None, None] * c0[None, :, None], W[:, None, None] * (1 - c0)[None, :, None]])
        assert np.max(np.abs(got - want)) <= 1e-5 * np.max(np.abs(want - b))


def test_site_map_and_column_arguments_are_checked():
    import torch
    with Simulation(LatticeParams(64, 8, **PARAMS), precision="dev32") as sim:
        for args in [(-1, 64), (64, 64), (0, 32)]:  # x0 out of range; a whole lattice narrower than the window
            with pytest.raises(capi.LBError) as e:
                sim.set_site_map(*args)
            assert e.value.code == capi.LB_ERR_BAD_PARAM
        buf = torch.empty((18, 8, 4), dtype=torch.float32, device="cuda")
        host = np.empty(18 * 8 * 4, np.float32)
        for x_first, n, ptr in [(61, 4, buf.data_ptr()), (-1, 4, buf.data_ptr()), (0, 0, buf.data_ptr()),
                                (0, 4, host.ctypes.data)]:
            with pytest.raises(capi.LBError) as e:
                capi.lb_export_columns(sim.h, 0, x_first, n, ptr)
            assert e.value.code == capi.LB_ERR_BAD_PARAM, (x_first, n)
        # a map that leaves the counters unchanged leaves the results unchanged
        sim.set_site_map(0, 64)
        sim.step(3)
        a = sim.populations()
    with Simulation(LatticeParams(64, 8, **PARAMS), precision="dev32") as sim:
        sim.step(3)
        np.testing.assert_array_equal(sim.populations(), a)
    with Simulation(LatticeParams(16, 8, **PARAMS)) as sim:
        sim.set_site_map(3, 32)
        with pytest.raises(capi.LBError) as e:
            sim.pressure_shift_gradient(10, 5)
        assert e.value.code == capi.LB_ERR_STATE
