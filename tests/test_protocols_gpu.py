"""The measurement protocols (the four-run non-equilibrium pressure of Sec. III.C, Eqs. EQP and
NEQP, and the seed-averaged structure factors of Appendix A) as the library runs them -- all runs
of a protocol in one batch, the final arithmetic on the returned averages -- against the same runs
of the oracle with the same seeds and noise stream (FP64 storage, so the two agree to rounding)."""
from dataclasses import replace

import numpy as np
import pytest

import oracle
from paper_1808_05168_gb300 import LatticeParams, protocols

pytestmark = pytest.mark.gpu

BASE = LatticeParams(32, 8, G=0.3, lambda_s=1.0, lambda_d=1.0, lambda_e=1.0)


def oracle_run(p, lattice_id, steps, discard, every):
    o = oracle.OracleLattice(p.Lx, p.Lz, lambda_s=p.lambda_s, lambda_d=p.lambda_d, lambda_e=p.lambda_e,
                             lambda_q=p.lambda_q, lambda_eps=p.lambda_eps, kT=p.kT, G=p.G, grad_c0=p.grad_c0,
                             seed=p.seed, lattice_id=lattice_id)
    o.set_sampling(discard, every)
    o.step(steps)
    return o


def test_ne_pressure_protocol_matches_the_oracle():
    """P_NE = P(kT, g) - P(0, g) - (P(kT, 0) - P(0, 0)) per seed, its mean and standard error, and
    the equilibrium shift, from the library's batch against the oracle's runs (the batch numbers
    its runs 0, 1, ... in the order: per seed (kT, g) then (kT, 0), then (0, g) and (0, 0))."""
    kT, g, seeds, steps, discard = 1e-4, 0.02, [7, 8, 9, 10], 600, 100
    r = protocols.ne_pressure(BASE, kT, g, seeds, steps, discard, every=10, precision="fp64")
    runs = []
    for s in seeds:
        runs += [replace(BASE, kT=kT, grad_c0=g, seed=s), replace(BASE, kT=kT, grad_c0=0.0, seed=s)]
    runs += [replace(BASE, kT=0.0, grad_c0=g), replace(BASE, kT=0.0, grad_c0=0.0)]
    P = np.array([oracle_run(p, i, steps, discard, 10).mean_pressure()[1] for i, p in enumerate(runs)])
    n = len(seeds)
    kg, k0 = P[0:2 * n:2], P[1:2 * n:2]
    per_seed = (kg - P[2 * n]) - (k0 - P[2 * n + 1])
    assert abs(r["P_ne"] - per_seed.mean()) <= 2e-12, (r["P_ne"], per_seed.mean())
    assert abs(r["stderr"] - per_seed.std(ddof=1) / np.sqrt(n)) <= 2e-12
    assert abs(r["dP_eq"] - (k0 - P[2 * n + 1]).mean()) <= 2e-12
    np.testing.assert_allclose([r["P_kT_grad"], r["P_0_grad"], r["P_kT_0"], r["P_0_0"]],
                               [kg.mean(), P[2 * n], k0.mean(), P[2 * n + 1]], rtol=1e-12, atol=0)


def test_seed_averaged_spectra_match_the_oracle():
    """Appendix A spectra of c and U_x averaged over four seeds, with their standard errors."""
    base = replace(BASE, kT=1e-4, grad_c0=0.02)
    seeds, steps, discard = [3, 4, 5, 6], 300, 50
    sp = protocols.ensemble_spectra(base, seeds, steps, discard, every=10, fields=("c", "ux"), precision="fp64")
    for f in ("c", "ux"):
        S = np.array([oracle_run(replace(base, seed=s), i, steps, discard, 10).structure_factor(f)[0]
                      for i, s in enumerate(seeds)])
        mean, err = S.mean(0), S.std(0, ddof=1) / np.sqrt(len(seeds))
        np.testing.assert_allclose(sp[f][0], mean, rtol=1e-9, atol=1e-12 * mean.max())
        np.testing.assert_allclose(sp[f][1], err, rtol=1e-6, atol=1e-12 * mean.max())
