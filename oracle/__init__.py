"""The oracle: a plain double-precision CPU implementation of the fluctuating two-species
D2Q9 lattice Boltzmann step of arXiv:1808.05168 (Sec. II, Eqs. LB, modes-discrete, bar,
aNI, ne-acc, MRT, noise-bin-expl, noise-bin-expl-high) and of its diagnostics (Sec. III.C
mean pressure; Appendix structure factors).

TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the benchmark's CPU
baseline are the only users; the product library never imports this package.  The C++
source (``lb_oracle.cpp``) is compiled with ``-O2 -ffp-contract=off`` so that every
operation rounds as written: once plain (``liblb_oracle.so``, one thread) and once with
``-fopenmp`` (``liblb_oracle_omp.so``), which runs the loops over the lattice rows on several
host cores and gives the same results bit for bit.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lb_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATHS = {False: os.path.join(_OUT_DIR, "liblb_oracle.so"),
              True: os.path.join(_OUT_DIR, "liblb_oracle_omp.so")}
_lock = threading.Lock()
_libs = {}


def build(force: bool = False, omp: bool = None) -> str:
    """Compile the oracle into ``oracle/_build/`` (host compiler only): the plain library, the
    OpenMP one, or both (omp=None, the default; returns the plain library's path)."""
    if omp is None:
        build(force, True)
        return build(force, False)
    path = _LIB_PATHS[omp]
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(path) and os.path.getmtime(path) >= os.path.getmtime(_SRC):
        return path
    tmp = path + f".tmp{os.getpid()}"
    cmd = (["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-fPIC", "-shared"] + (["-fopenmp"] if omp else [])
           + ["-o", tmp, _SRC])
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def _load(omp: bool = False):
    with _lock:
        if omp in _libs:
            return _libs[omp]
        lib = ctypes.CDLL(build(omp=omp))
        c_dbl, c_int, c_i64, c_u64, c_u32, vp = (ctypes.c_double, ctypes.c_int, ctypes.c_int64,
                                                  ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p)
        dp = ctypes.POINTER(ctypes.c_double)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        create_args = [c_int, c_int, c_dbl, c_dbl, c_dbl, c_dbl, c_dbl, c_dbl, c_dbl, c_dbl, c_u64, c_u32,
                       c_int, c_int, c_int]
        lib.olb_create.argtypes = create_args
        lib.olb_create.restype = vp
        lib.olb_destroy.argtypes = [vp]
        lib.olb_set_sampling.argtypes = [vp, c_i64, c_i64]
        lib.olb_step.argtypes = [vp, c_i64]
        lib.olb_time.argtypes = [vp]
        lib.olb_time.restype = c_i64
        lib.olb_set_time.argtypes = [vp, c_i64]
        lib.olb_set_site_map.argtypes = [vp, c_int, c_int]
        lib.olb_get_populations.argtypes = [vp, dp]
        lib.olb_set_populations.argtypes = [vp, dp]
        lib.olb_mass.argtypes = [vp, dp]
        lib.olb_fields.argtypes = [vp, dp]
        lib.olb_structure_factor.argtypes = [vp, c_int, dp]
        lib.olb_structure_factor.restype = c_i64
        lib.olb_set_correlations.argtypes = [vp, c_int, c_int, ctypes.POINTER(c_int)]
        lib.olb_correlation.argtypes = [vp, c_int, dp]
        lib.olb_correlation.restype = c_i64
        lib.olb_mode_correlation.argtypes = [vp, c_int, c_int, dp]
        lib.olb_mode_correlation.restype = c_i64
        lib.olb_profile.argtypes = [vp, c_int, dp]
        lib.olb_profile.restype = c_i64
        lib.olb_mean_pressure.argtypes = [vp, dp, dp]
        lib.olb_mean_pressure.restype = c_i64
        lib.olb_site_noise.argtypes = [vp, c_int, c_int, c_i64, dp]
        lib.olb_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.olb_site_normals.argtypes = [c_u64, c_u32, c_u32, c_u32, dp]
        lib.olb_box_muller.argtypes = [u32p, c_i64, dp]
        lib.olb_basis.argtypes = [dp, dp, dp]
        lib.olb_dft2_power.argtypes = [dp, c_int, c_int, dp]
        lib.olb_pressure_shift_grad.argtypes = create_args + [c_i64, dp, dp]
        lib.olb_pressure_shift.argtypes = create_args + [c_i64]
        lib.olb_pressure_shift.restype = c_dbl
        lib.olb_set_threads.argtypes = [c_int]
        lib.olb_set_threads.restype = c_int
        _libs[omp] = lib
        return lib


def set_threads(n: int = 0) -> int:
    """Threads of the OpenMP oracle's row loops (n > 0 sets them); returns the count in use."""
    return int(_load(True).olb_set_threads(int(n)))


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


FIELDS = {"rho": 0, "c": 1, "ux": 2, "uz": 3}
PROFILE_FIELDS = {"rho": 0, "c": 1, "ux": 2, "uz": 3, "p": 4}


class OracleLattice:
    """One lattice of the oracle.  Parameters follow the paper's statement of the problem
    (Sec. II.A): Lx x Lz sites, relaxation rates (lambda_s, lambda_d, lambda_e, lambda_Q,
    lambda_eps), thermal energy kT, coupling G and imposed gradient grad_c0."""

    def __init__(self, Lx, Lz, lambda_s=1.0, lambda_d=0.8, lambda_e=None, lambda_q=1.0, lambda_eps=1.0,
                 kT=0.0, G=0.0, grad_c0=0.0, seed=1, lattice_id=0, astar=True, wall_fixed=False,
                 noise_loc=False, omp=False):
        """omp: run on the OpenMP build (the row loops on several host cores, same results)."""
        self.lib = _load(omp)
        if lambda_e is None:
            lambda_e = lambda_s
        self.Lx, self.Lz = int(Lx), int(Lz)
        self.params = dict(lambda_s=lambda_s, lambda_d=lambda_d, lambda_e=lambda_e, lambda_q=lambda_q,
                           lambda_eps=lambda_eps, kT=kT, G=G, grad_c0=grad_c0, seed=seed,
                           lattice_id=lattice_id, astar=astar, wall_fixed=wall_fixed, noise_loc=noise_loc)
        self.h = self.lib.olb_create(self.Lx, self.Lz, lambda_s, lambda_d, lambda_e, lambda_q, lambda_eps, kT, G,
                                     grad_c0, seed, lattice_id, int(astar), int(wall_fixed), int(noise_loc))
        if not self.h:
            raise ValueError("oracle: bad lattice size")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.olb_destroy(h)
            self.h = None

    @property
    def n_sites(self):
        return self.Lx * self.Lz

    def set_sampling(self, discard, every):
        self.lib.olb_set_sampling(self.h, int(discard), int(every))

    def step(self, n=1):
        self.lib.olb_step(self.h, int(n))

    @property
    def time(self):
        return int(self.lib.olb_time(self.h))

    @time.setter
    def time(self, t):
        self.lib.olb_set_time(self.h, int(t))

    def set_site_map(self, x0, Lx_global):
        """Use the noise counters of columns x0.. of a lattice Lx_global wide (window checks)."""
        self.lib.olb_set_site_map(self.h, int(x0), int(Lx_global))

    def populations(self) -> np.ndarray:
        out = np.empty((2, 9, self.Lz, self.Lx), np.float64)
        self.lib.olb_get_populations(self.h, _dptr(out))
        return out

    def set_populations(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(2, 9, self.Lz, self.Lx)
        self.lib.olb_set_populations(self.h, _dptr(f))

    def mass(self):
        out = np.empty(2, np.float64)
        self.lib.olb_mass(self.h, _dptr(out))
        return out

    def fields(self):
        """Pre-collision fields of the next step: dict of rhoA, rhoB, ux, uz, p ([Lz, Lx])."""
        out = np.empty((5, self.Lz, self.Lx), np.float64)
        self.lib.olb_fields(self.h, _dptr(out))
        return dict(rhoA=out[0], rhoB=out[1], ux=out[2], uz=out[3], p=out[4])

    def structure_factor(self, field):
        out = np.empty((self.Lz, self.Lx), np.float64)
        n = self.lib.olb_structure_factor(self.h, FIELDS[field] if isinstance(field, str) else int(field),
                                          _dptr(out))
        return out, int(n)

    def profile(self, field):
        """Time average over the samples of the row means of rho, c, Ux, Uz or P (Sec. III.C
        profiles), rows 0..Lz-1, and the sample count."""
        out = np.empty(self.Lz, np.float64)
        k = PROFILE_FIELDS[field] if isinstance(field, str) else int(field)
        n = self.lib.olb_profile(self.h, k, _dptr(out))
        return out, int(n)

    def set_correlations(self, fields, modes=()):
        """Accumulate, from the next sample on, the equal-x real-space correlation of each field in
        `fields` and its mode correlations C(q_x, z, z') for the q_x mode indices `modes`."""
        mask = 0
        for f in fields:
            mask |= 1 << (FIELDS[f] if isinstance(f, str) else int(f))
        m = (ctypes.c_int * max(1, len(modes)))(*[int(k) for k in modes])
        self.modes = list(modes)
        self.lib.olb_set_correlations(self.h, mask, len(modes), m)

    def correlation(self, field):
        """<dphi(x, z) dphi(x, z')> averaged over x and the samples: (Lz, Lz) array, sample count."""
        out = np.empty((self.Lz, self.Lz), np.float64)
        n = self.lib.olb_correlation(self.h, FIELDS[field] if isinstance(field, str) else int(field), _dptr(out))
        return out, int(n)

    def mode_correlation(self, field, mode_index):
        """C(q_x, z, z') = <dphi(q_x, z)^* dphi(q_x, z')> for the mode_index-th requested mode."""
        out = np.empty((self.Lz, self.Lz, 2), np.float64)
        n = self.lib.olb_mode_correlation(self.h, FIELDS[field] if isinstance(field, str) else int(field),
                                          int(mode_index), _dptr(out))
        return out[..., 0] + 1j * out[..., 1], int(n)

    def mean_pressure(self):
        last = ctypes.c_double()
        avg = ctypes.c_double()
        n = self.lib.olb_mean_pressure(self.h, ctypes.byref(last), ctypes.byref(avg))
        return last.value, avg.value, int(n)

    def site_noise(self, x, z, step):
        out = np.empty(18, np.float64)
        self.lib.olb_site_noise(self.h, int(x), int(z), int(step), _dptr(out))
        return out.reshape(2, 9)


def philox4x32_10(ctr, key):
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib.olb_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def site_normals(seed, lattice_id, site, step):
    lib = _load()
    out = np.empty(16, np.float64)
    lib.olb_site_normals(int(seed), int(lattice_id), int(site), int(step), _dptr(out))
    return out


def box_muller(words) -> np.ndarray:
    """Box-Muller normals in FP64 of the word pairs (words[2i], words[2i+1]), in that order."""
    lib = _load()
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint32).reshape(-1))
    if w.size % 2:
        raise ValueError("words must hold pairs")
    out = np.empty(w.size, np.float64)
    lib.olb_box_muller(w.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), w.size // 2, _dptr(out))
    return out


def basis():
    lib = _load()
    T = np.empty((9, 9), np.float64)
    w = np.empty(9, np.float64)
    N = np.empty(9, np.float64)
    lib.olb_basis(_dptr(T), _dptr(w), _dptr(N))
    return T, w, N


def dft2_power(phi: np.ndarray, omp: bool = False):
    """The O(n^2) separable transform's power |phi(q)|^2 / (Lx Lz), [q_z][q_x]; omp: on the
    OpenMP build (its rows and columns on every host core; same result)."""
    lib = _load(omp)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    Lz, Lx = phi.shape
    out = np.empty_like(phi)
    lib.olb_dft2_power(_dptr(phi), int(Lx), int(Lz), _dptr(out))
    return out


def _lattice_args(Lx, Lz, lambda_s, lambda_d, lambda_e, lambda_q, lambda_eps, kT, G, grad_c0, seed, lattice_id,
                  astar, wall_fixed, noise_loc):
    if lambda_e is None:
        lambda_e = lambda_s
    return (int(Lx), int(Lz), float(lambda_s), float(lambda_d), float(lambda_e), float(lambda_q),
            float(lambda_eps), float(kT), float(G), float(grad_c0), int(seed), int(lattice_id), int(astar),
            int(wall_fixed), int(noise_loc))


def pressure_shift(Lx, Lz, nsteps, lambda_s=1.0, lambda_d=0.8, lambda_e=None, lambda_q=1.0, lambda_eps=1.0,
                   kT=1e-5, G=0.5, grad_c0=0.0, seed=5, lattice_id=0, astar=True, wall_fixed=False,
                   noise_loc=False):
    """Loss (1/n) sum_t Pbar(t) at kT minus the same at kT = 0, from the rest state."""
    lib = _load()
    args = _lattice_args(Lx, Lz, lambda_s, lambda_d, lambda_e, lambda_q, lambda_eps, kT, G, grad_c0, seed,
                         lattice_id, astar, wall_fixed, noise_loc)
    return float(lib.olb_pressure_shift(*args, int(nsteps)))


def pressure_shift_grad(Lx, Lz, nsteps, lambda_s=1.0, lambda_d=0.8, lambda_e=None, lambda_q=1.0,
                        lambda_eps=1.0, kT=1e-5, G=0.5, grad_c0=0.0, seed=5, lattice_id=0, astar=True,
                        wall_fixed=False, noise_loc=False):
    """(loss, [dL/dG, dL/dlambda_s, dL/dlambda_d]) by forward-mode dual numbers."""
    lib = _load()
    args = _lattice_args(Lx, Lz, lambda_s, lambda_d, lambda_e, lambda_q, lambda_eps, kT, G, grad_c0, seed,
                         lattice_id, astar, wall_fixed, noise_loc)
    loss = ctypes.c_double()
    grad = np.empty(3, np.float64)
    lib.olb_pressure_shift_grad(*args, int(nsteps), ctypes.byref(loss), _dptr(grad))
    return loss.value, grad


def _sampled_run(job):
    """One oracle lattice run with sampling (a worker of sampled_runs): its structure factors."""
    kwargs, Lx, Lz, steps, discard, every, fields = job
    o = OracleLattice(Lx, Lz, **kwargs)
    o.set_sampling(discard, every)
    o.step(steps)
    return {f: o.structure_factor(f) for f in fields}


def sampled_runs(jobs, processes=None):
    """Independent oracle runs, one per job (kwargs of OracleLattice, Lx, Lz, steps, discard,
    every, fields), in a pool of spawned processes (plain build, one thread each); returns, per
    job, {field: (S(q_z, q_x) average, sample count)}."""
    import multiprocessing as mp

    build()
    with mp.get_context("spawn").Pool(processes or os.cpu_count() or 1) as pool:
        return pool.map(_sampled_run, list(jobs))
