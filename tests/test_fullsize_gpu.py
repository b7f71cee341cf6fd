"""Parity at the benchmark's full sizes and launch configuration.

The ensemble (768 lattices, 66.8 M sites) runs exactly as the benchmark times it (FP32
deviations, CUDA graphs, autotuned tile); a set of its lattices is then compared in full with
the oracle run from the same rest state.  The 8192 x 2048 lattice is checked one step at a time
on column windows: a site's update depends only on the state within two columns, so the oracle
on a 5-column window (with the large lattice's noise counters) gives that column exactly.
"""
import numpy as np
import pytest

import oracle
from paper_1808_05168_gb300 import Simulation, workloads

pytestmark = pytest.mark.gpu

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def background(Lx, Lz, grad_c0):
    z = np.arange(Lz) + 0.5 - Lz / 2
    c0 = 0.5 + z * grad_c0
    b = np.empty((2, 9, Lz, Lx))
    for l in range(9):
        b[0, l] = (W[l] * c0)[:, None]
        b[1, l] = (W[l] * (1 - c0))[:, None]
    return b


def oracle_of(p, Lx=None):
    return oracle.OracleLattice(Lx or p.Lx, p.Lz, lambda_s=p.lambda_s, lambda_d=p.lambda_d, lambda_e=p.lambda_e,
                                lambda_q=p.lambda_q, lambda_eps=p.lambda_eps, kT=p.kT, G=p.G, grad_c0=p.grad_c0,
                                seed=p.seed, lattice_id=p.lattice_id)


def test_ensemble_in_benchmark_configuration():
    lattices = workloads.c3()
    steps = 12
    with Simulation(lattices, precision="dev32", graph=True, autotune=True) as sim:
        sim.set_sampling(0, 100)
        sim.step(steps)
        picks = [0, 1, 2, 5, 10, 11, 383, 766, 767]  # every size, every gradient, both ends of the ids
        got = {i: sim.populations(i) for i in picks}
    for i in picks:
        p = lattices[i]
        o = oracle_of(p)
        o.step(steps)
        want = o.populations()
        dev = want - background(p.Lx, p.Lz, p.grad_c0)
        err = np.max(np.abs(got[i] - want))
        assert err <= 1e-5 * np.max(np.abs(dev)), (i, err, np.max(np.abs(dev)))


@pytest.mark.parametrize("prec", ["dev32", "fp64"])
def test_large_lattice_column_windows(prec):
    (p,) = workloads.c4()
    Lx, Lz = p.Lx, p.Lz
    cols = [0, 1, 127, 128, 4095, 8190, 8191]
    with Simulation(p, precision=prec, autotune=True) as sim:
        sim.step(2)
        before = sim.populations()
        sim.step(1)
        after = sim.populations()
    b = background(5, Lz, p.grad_c0)
    for x in cols:
        idx = [(x + d) % Lx for d in range(-2, 3)]
        o = oracle_of(p, Lx=5)
        o.set_site_map((x - 2) % Lx, Lx)
        o.set_populations(before[:, :, :, idx])
        o.time = 2
        o.step(1)
        want = o.populations()[:, :, :, 2]
        got = after[:, :, :, x]
        if prec == "fp64":
            rel = np.max(np.abs(got - want) / np.abs(want))
            assert rel <= 1e-12, (x, rel)
        else:
            dev = np.max(np.abs(o.populations() - b))
            err = np.max(np.abs(got - want))
            assert err <= 1e-5 * dev, (x, err, dev)
