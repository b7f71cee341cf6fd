"""Synthetic workloads of the benchmark and the tests, as parameter recipes only (no
arithmetic of the method lives here).  All inputs are generated: the initial state is the
method's rest state, and the noise is the seeded Philox stream.

  c1  64 x 32 ideal mixture (G = 0), kT = 1e-5, wall-to-wall difference 0.5, seed 1
  c2  512 x 256 non-ideal mixture, G = 0.5, gradient 0.5 / Lz, kT = 1e-5, seed 2
  c3  ensemble: 64 seeds x Lz in {32, 64, 128, 256} (Lx = 4 Lz) x difference in
      {0.1, 0.3, 0.5}, G = 0.5, kT = 1e-5: 768 lattices, 66,846,720 sites
  c4  8192 x 2048 non-ideal mixture, G = 0.5, difference 0.5, kT = 1e-5, seed 4
  c5  256 x 128 non-ideal mixture, G = 0.5, difference 0.5, kT = 1e-5, seed 5 (gradients)

Relaxation rates follow the reading of "1.0 for shear and 0.8 for diffusion" as rates:
lambda_s = lambda_e = 1.0, lambda_d = 0.8, lambda_Q = lambda_eps = 1.0.
"""
from __future__ import annotations

from . import LatticeParams

RATES = dict(lambda_s=1.0, lambda_d=0.8, lambda_e=1.0, lambda_q=1.0, lambda_eps=1.0)


def c1():
    return [LatticeParams(64, 32, kT=1e-5, G=0.0, grad_c0=0.5 / 32, seed=1, **RATES)]


def c2():
    return [LatticeParams(512, 256, kT=1e-5, G=0.5, grad_c0=0.5 / 256, seed=2, **RATES)]


def c3(n_seeds: int = 64, sizes=(32, 64, 128, 256), deltas=(0.1, 0.3, 0.5), seed0: int = 1000, id0: int = 0):
    out = []
    lid = id0
    for s in range(n_seeds):
        for L in sizes:
            for dc in deltas:
                out.append(LatticeParams(4 * L, L, kT=1e-5, G=0.5, grad_c0=dc / L, seed=seed0 + s, lattice_id=lid,
                                         **RATES))
                lid += 1
    return out


def c4():
    return [LatticeParams(8192, 2048, kT=1e-5, G=0.5, grad_c0=0.5 / 2048, seed=4, **RATES)]


def c5():
    return [LatticeParams(256, 128, kT=1e-5, G=0.5, grad_c0=0.5 / 128, seed=5, **RATES)]


def sites(lattices) -> int:
    return sum(p.Lx * p.Lz for p in lattices)
