"""The multi-rank path on CPU: two gloo ranks each run their own seeds of a small ensemble (the
oracle stands in for the per-rank work) and combine the ensemble average on the host; the result
equals the single-process average over all seeds."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

import oracle
from paper_1808_05168_gb300.ensemble import ensemble_mean, seeds_for_rank

N_PER_RANK = 2


def spectra_sum(seeds):
    tot = None
    for s in seeds:
        o = oracle.OracleLattice(8, 4, kT=1e-4, G=0.3, grad_c0=0.02, seed=s, lattice_id=0)
        o.set_sampling(10, 5)
        o.step(60)
        S, _ = o.structure_factor("c")
        P = o.mean_pressure()[1]
        v = np.concatenate([S.ravel(), [P]])
        tot = v if tot is None else tot + v
    return tot


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seeds = seeds_for_rank(rank, N_PER_RANK)
    mean = ensemble_mean(spectra_sum(seeds), len(seeds))
    out[rank] = mean.tolist()
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_combine_to_the_serial_ensemble_average():
    oracle.build()
    world = 2
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = [np.array(out[r]) for r in range(world)]
    np.testing.assert_array_equal(res[0], res[1])
    all_seeds = [s for r in range(world) for s in seeds_for_rank(r, N_PER_RANK)]
    assert len(set(all_seeds)) == world * N_PER_RANK
    serial = spectra_sum(all_seeds) / len(all_seeds)
    np.testing.assert_allclose(res[0], serial, rtol=1e-13, atol=0)
