"""Measurement protocols of the paper built on the C interface (argument marshalling and the
final arithmetic on returned averages only; every step runs in the CUDA library).

- ``ne_pressure``: the non-equilibrium part of the spatially averaged pressure by the four-run
  protocol of Sec. III.C, Eqs. (EQP) and (NEQP):
      dP_eq  = Pbar(L, kT, 0)        - Pbar(L, 0, 0)
      Pbar_NE = Pbar(L, kT, grad c0) - Pbar(L, 0, grad c0) - dP_eq,
  with the kT > 0 runs averaged over independent seeds, all runs advanced together in one batch.
- ``ensemble_spectra``: structure factors (Appendix A) averaged over seeds of one configuration.
"""
from __future__ import annotations

from dataclasses import replace

import numpy as np

from . import LatticeParams, Simulation


def _batch_ids(lattices):
    return [replace(p, lattice_id=i) for i, p in enumerate(lattices)]


def ne_pressure(base: LatticeParams, kT: float, grad_c0: float, seeds, steps: int, discard: int,
                every: int = 10, precision: str = "dev32"):
    """Pbar_NE (Eq. NEQP) for one (L, kT, grad_c0) with its standard error over the seeds.
    Returns dict(P_ne, stderr, dP_eq, P_kT_grad, P_0_grad, P_kT_0, P_0_0)."""
    seeds = list(seeds)
    runs = []
    for s in seeds:
        runs.append(replace(base, kT=kT, grad_c0=grad_c0, seed=s))
        runs.append(replace(base, kT=kT, grad_c0=0.0, seed=s))
    runs.append(replace(base, kT=0.0, grad_c0=grad_c0))
    runs.append(replace(base, kT=0.0, grad_c0=0.0))
    runs = _batch_ids(runs)
    with Simulation(runs, precision=precision) as sim:
        sim.set_sampling(discard, every)
        sim.step(steps)
        P = np.array([sim.mean_pressure(i)[1] for i in range(len(runs))])
    n = len(seeds)
    P_kg, P_k0 = P[0:2 * n:2], P[1:2 * n:2]
    P_0g, P_00 = P[2 * n], P[2 * n + 1]
    per_seed = (P_kg - P_0g) - (P_k0 - P_00)
    return dict(P_ne=float(per_seed.mean()), stderr=float(per_seed.std(ddof=1) / np.sqrt(n)) if n > 1 else float("nan"),
                dP_eq=float((P_k0 - P_00).mean()), P_kT_grad=float(P_kg.mean()), P_0_grad=float(P_0g),
                P_kT_0=float(P_k0.mean()), P_0_0=float(P_00))


def ne_pressure_scan(base: LatticeParams, kT: float, grads, seeds, steps: int, discard: int, every: int = 10,
                     precision: str = "dev32"):
    """Pbar_NE (Eq. NEQP) for several gradients at one (L, kT) in one batch, the equilibrium
    companions (kT, grad 0) and (0, 0) shared.  Returns a list of dict(grad_c0, P_ne, stderr)."""
    seeds = list(seeds)
    grads = list(grads)
    runs = []
    for s in seeds:
        runs += [replace(base, kT=kT, grad_c0=g, seed=s) for g in grads]
        runs.append(replace(base, kT=kT, grad_c0=0.0, seed=s))
    runs += [replace(base, kT=0.0, grad_c0=g) for g in grads]
    runs.append(replace(base, kT=0.0, grad_c0=0.0))
    runs = _batch_ids(runs)
    m = len(grads) + 1
    with Simulation(runs, precision=precision) as sim:
        sim.set_sampling(discard, every)
        sim.step(steps)
        P = np.array([sim.mean_pressure(i)[1] for i in range(len(runs))])
    n = len(seeds)
    noisy = P[: n * m].reshape(n, m)
    quiet = P[n * m:]
    out = []
    for k, g in enumerate(grads):
        per_seed = (noisy[:, k] - quiet[k]) - (noisy[:, -1] - quiet[-1])
        out.append(dict(grad_c0=g, P_ne=float(per_seed.mean()),
                        stderr=float(per_seed.std(ddof=1) / np.sqrt(n)) if n > 1 else float("nan")))
    return out


def ensemble_spectra(base: LatticeParams, seeds, steps: int, discard: int, every: int = 10,
                     fields=("rho", "c", "ux", "uz"), precision: str = "dev32"):
    """Structure factors S(q_z, q_x) averaged over seeds (one batch).  Returns {field: (mean,
    stderr)} with arrays of shape (Lz, Lx)."""
    runs = _batch_ids([replace(base, seed=s) for s in seeds])
    out = {}
    with Simulation(runs, precision=precision) as sim:
        sim.set_sampling(discard, every)
        sim.step(steps)
        for f in fields:
            S = np.array([sim.structure_factor(f, lattice=i)[0] for i in range(len(runs))])
            out[f] = (S.mean(axis=0), S.std(axis=0, ddof=1) / np.sqrt(len(runs)) if len(runs) > 1 else 0 * S[0])
    return out


def ensemble_correlations(base: LatticeParams, seeds, steps: int, discard: int, every: int = 10,
                          fields=("c", "ux"), precision: str = "dev32"):
    """Real-space correlations <dphi(x, z) dphi(x, z')>_x averaged over seeds (one batch).
    Returns {field: (mean, stderr)} with arrays of shape (Lz, Lz)."""
    runs = _batch_ids([replace(base, seed=s) for s in seeds])
    out = {}
    with Simulation(runs, precision=precision) as sim:
        sim.set_sampling(discard, every)
        sim.set_correlations(fields)
        sim.step(steps)
        for f in fields:
            R = np.array([sim.correlation(f, lattice=i)[0] for i in range(len(runs))])
            out[f] = (R.mean(axis=0), R.std(axis=0, ddof=1) / np.sqrt(len(runs)) if len(runs) > 1 else 0 * R[0])
    return out
