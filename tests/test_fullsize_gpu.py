"""Parity at the benchmark's full sizes and launch configuration.

The ensemble (768 lattices, 66.8 M sites) runs exactly as the benchmark times it (FP32
deviations, CUDA graphs, the persistent launch of the plain steps, autotuned tile, a sample every
100 steps, advanced one sample step and 99 plain steps at a time); a set of its lattices is then
compared in full with the oracle run from the same rest state.  The 8192 x 2048 lattice is checked one step at a time
on column windows: a site's update depends only on the state within two columns, so the oracle
on a 5-column window (with the large lattice's noise counters) gives that column exactly.
"""
import numpy as np
import pytest

import oracle
from paper_1808_05168_gb300 import LatticeParams, Simulation, workloads

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


def oracle_of(p, Lx=None, omp=False):
    return oracle.OracleLattice(Lx or p.Lx, p.Lz, lambda_s=p.lambda_s, lambda_d=p.lambda_d, lambda_e=p.lambda_e,
                                lambda_q=p.lambda_q, lambda_eps=p.lambda_eps, kT=p.kT, G=p.G, grad_c0=p.grad_c0,
                                seed=p.seed, lattice_id=p.lattice_id, omp=omp)


def test_ensemble_in_benchmark_configuration():
    """201 steps as the benchmark runs them: sample steps 0, 100 and 200 (ordinary launches with
    their diagnostics kernels), each of the two runs of 99 plain steps in between one persistent
    launch (items of the autotuned tile handed out in order, per-item dependency waits), all in
    CUDA graphs.  Lattices of every size and gradient and both ends of the ids against the
    oracle: populations (1e-5 of the deviations), S_c(q_x, q_z) and the other three fields'
    spectra over the whole q grid (the bar of the spectra tests), and the mean pressure (1e-7)."""
    lattices = workloads.c3()
    with Simulation(lattices, precision="dev32", graph=True, persistent=True, autotune=True) as sim:
        sim.set_sampling(0, 100)
        for _ in range(2):
            sim.step(1)
            sim.step(99)
        sim.step(1)
        assert sim.time == 201
        picks = [0, 2, 5, 8, 11, 383, 766]  # every size, every gradient, both ends of the ids
        got = {i: (sim.populations(i), {f: sim.structure_factor(f, lattice=i) for f in ("rho", "c", "ux", "uz")},
                   sim.mean_pressure(i)) for i in picks}
    for i in picks:
        p = lattices[i]
        o = oracle_of(p, omp=True)
        o.set_sampling(0, 100)
        o.step(201)
        want = o.populations()
        dev = want - background(p.Lx, p.Lz, p.grad_c0)
        f32, S, (last, avg) = got[i]
        err = np.max(np.abs(f32 - want))
        assert err <= 1e-5 * np.max(np.abs(dev)), (i, err, np.max(np.abs(dev)))
        for f, (Sg, n) in S.items():
            Sw, no = o.structure_factor(f)
            assert n == no == 3, (i, f, n, no)
            # absolute part: the noise-dominated modes; relative part: the q_x = 0 modes, which carry
            # the deterministic density and concentration profiles -- the FP32 deviations behind
            # them carry the populations' bar (1e-5), doubled in |phi(q)|^2, plus FP32 transforms
            err = np.abs(Sg - Sw)
            assert np.all(err <= 2e-3 * Sw.mean() + 5e-5 * np.abs(Sw)), (
                i, f, float(np.max(err / (2e-3 * Sw.mean() + 5e-5 * np.abs(Sw)))), float(np.max(err / np.abs(Sw).max())))
        olast, oavg, _ = o.mean_pressure()
        assert abs(last - olast) <= 1e-7 * abs(olast) and abs(avg - oavg) <= 1e-7 * abs(oavg), (i, last, olast)


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


@pytest.fixture(scope="module")
def c2_oracle():
    (p,) = workloads.c2()
    o = oracle_of(p, omp=True)
    o.set_sampling(40, 10)
    o.step(60)
    return p, o


@pytest.mark.parametrize("prec", ["fp64", "dev32"])
def test_c2_spectra_pressure_and_profiles(prec, c2_oracle):
    """The 512 x 256 lattice (G = 0.5, wall-to-wall difference 0.5, kT = 1e-5) with the
    diagnostics of Appendix A and Sec. III.C on two sample steps: every field's S(q_x, q_z) over
    the whole q grid, the mean pressure and the z-profiles, against the oracle."""
    p, o = c2_oracle
    with Simulation(p, precision=prec, graph=True) as sim:
        sim.set_sampling(40, 10)
        sim.step(60)
        S = {f: sim.structure_factor(f) for f in ("rho", "c", "ux", "uz")}
        last, avg = sim.mean_pressure()
        prof = {f: sim.profile(f) for f in ("rho", "c", "ux", "uz", "p")}
    for f, (got, n) in S.items():
        want, no = o.structure_factor(f)
        assert n == no == 2
        if prec == "fp64":
            np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-12 * want.max())
        else:
            # absolute part: the noise-dominated modes; relative part: the q_x = 0 modes, which
            # carry the deterministic density and concentration profiles (FP32 row sums)
            assert np.all(np.abs(got - want) <= 2e-3 * want.mean() + 1e-5 * np.abs(want)), f
    olast, oavg, _ = o.mean_pressure()
    tol = 1e-12 if prec == "fp64" else 1e-7
    assert abs(last - olast) <= tol * abs(olast) and abs(avg - oavg) <= tol * abs(oavg)
    z = np.arange(p.Lz) + 0.5 - p.Lz / 2
    bg = {"rho": 1.0, "c": 0.5 + z * p.grad_c0, "ux": 0.0, "uz": 0.0}
    for f, (got, n) in prof.items():
        want, _ = o.profile(f)
        if prec == "fp64":
            np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15)
        else:
            b = bg.get(f, want.mean())
            assert np.max(np.abs(got - want)) <= 1e-5 * np.max(np.abs(want - b)) + 1e-12, f


@pytest.mark.parametrize("prec,kw", [("dev32", dict(persistent=True)), ("fp64", dict())], ids=["dev32", "fp64"])
def test_largest_lattices_in_one_batch(prec, kw):
    """The largest lattice the interface admits (18 Lx Lz just below 2^31 values: 32768 x 3640,
    119 M sites) twice in one batch, so that the second lattice's populations start beyond 2^31
    values (64-bit offsets in the batch, per-lattice tensor maps) -- 34 GB of FP32 or 69 GB of FP64
    state.  One step from rest, then one more: column windows at both x edges and in the middle of
    both lattices against the oracle (a site's update depends only on the state within two columns,
    so the oracle on a 5-column window with the large lattice's noise counters gives that column
    exactly)."""
    import torch
    Lx, Lz = 32768, 3640
    assert 18 * Lx * Lz < 2 ** 31
    ps = [LatticeParams(Lx, Lz, kT=1e-5, G=0.5, grad_c0=0.5 / Lz, seed=41, lattice_id=i,
                        lambda_s=1.0, lambda_d=0.8, lambda_e=1.0) for i in range(2)]
    cols = [0, 1, 16383, 32766, 32767]
    # (each lattice's populations are 17 GB in double precision on the host: keep only the windows)
    windows = lambda f: {x: np.ascontiguousarray(f[..., [(x + d) % Lx for d in range(-2, 3)]]) for x in cols}
    with Simulation(ps, precision=prec, **kw) as sim:
        sim.step(1)
        before = [windows(sim.populations(i)) for i in range(2)]
        sim.step(1)
        after = [{x: np.ascontiguousarray(f[..., x]) for x in cols} for f in (sim.populations(i) for i in range(2))]
    torch.cuda.empty_cache()
    b = background(5, Lz, ps[0].grad_c0)
    for i, p in enumerate(ps):
        for x in cols:
            o = oracle_of(p, Lx=5)
            o.set_site_map((x - 2) % Lx, Lx)
            o.set_populations(before[i][x])
            o.time = 1
            o.step(1)
            want = o.populations()[:, :, :, 2]
            got = after[i][x]
            if prec == "fp64":
                assert np.max(np.abs(got - want) / np.abs(want)) <= 1e-12, (i, x)
            else:
                assert np.max(np.abs(got - want)) <= 1e-5 * np.max(np.abs(o.populations() - b)), (i, x)
