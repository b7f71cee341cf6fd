"""GB300 (sm_103a) implementation of the fluctuating two-species D2Q9 lattice Boltzmann method
of Belardinelli, Sbragaglia, Benzi & Ciliberto (arXiv:1808.05168): the fused per-step update
(Eq. LB with Eq. MRT, forces of Eqs. aNI and ne-acc, FDT noise of Eqs. noise-bin-expl and
noise-bin-expl-high, mid-way bounce-back walls of Sec. II.A) and its diagnostics (structure
factors of Appendix A, mean pressure of Sec. III.C).

All arithmetic runs in the CUDA library behind ``include/lb.h``; this package only marshals
arguments (``capi``) and offers a small object wrapper (:class:`Simulation`).
"""
from __future__ import annotations

from dataclasses import dataclass, field as dc_field

import numpy as np

from . import capi
from .capi import LBError

__all__ = ["LatticeParams", "Simulation", "LBError", "capi"]


@dataclass
class LatticeParams:
    """One lattice: size, relaxation rates (Eq. MRT, Table I), kT, coupling G (Eq. aNI),
    imposed gradient grad_c0 (Eq. ne-acc), and the Philox key/counter words of its noise."""
    Lx: int
    Lz: int
    lambda_s: float = 1.0
    lambda_d: float = 0.8
    lambda_e: float | None = None   # defaults to lambda_s
    lambda_q: float = 1.0
    lambda_eps: float = 1.0
    kT: float = 0.0
    G: float = 0.0
    grad_c0: float = 0.0
    seed: int = 1
    lattice_id: int = 0

    def to_c(self) -> capi.lb_params:
        le = self.lambda_s if self.lambda_e is None else self.lambda_e
        return capi.lb_params(int(self.Lx), int(self.Lz), float(self.lambda_s), float(self.lambda_d), float(le),
                              float(self.lambda_q), float(self.lambda_eps), float(self.kT), float(self.G),
                              float(self.grad_c0), int(self.seed), int(self.lattice_id), 0)


FIELDS = {"rho": capi.LB_FIELD_RHO, "c": capi.LB_FIELD_C, "ux": capi.LB_FIELD_UX, "uz": capi.LB_FIELD_UZ,
          "p": capi.LB_FIELD_P}


class Simulation:
    """A batch of lattices advanced together on the GPU (a single lattice is a batch of one)."""

    def __init__(self, lattices, precision: str = "fp64", astar: bool = True, wall_fixed: bool = False,
                 noise_loc: bool = False, graph: bool = False, persistent: bool = False, autotune: bool = False,
                 bulk: bool = True, tensor_maps: bool = True, allocator=None):
        """precision: "fp64" (FP64 populations) or "dev32" (FP32 deviations from the background).
        graph: lb_step through captured CUDA graphs; persistent: one cooperative launch per run of
        plain steps (items handed out in order, each waiting only for its neighbours' previous
        step), the fastest launch for batches; autotune: time tile shapes on the first step.
        bulk / tensor_maps: stage rows with bulk copies / with 3-d tensor copies of link runs
        (FP32) where possible (both default; results are bit-identical either way).
        allocator: None (the library allocates with cudaMalloc), "torch" (torch's caching
        allocator on the current device) or an (alloc, free) pair of capi callbacks."""
        if isinstance(lattices, LatticeParams):
            lattices = [lattices]
        self.lattices = list(lattices)
        flags = {"fp64": capi.LB_PREC_FP64, "dev32": capi.LB_PREC_DEV32}[precision]
        flags |= 0 if astar else capi.LB_NO_ASTAR
        flags |= capi.LB_WALL_FIXED if wall_fixed else 0
        flags |= capi.LB_NOISE_LOC if noise_loc else 0
        flags |= capi.LB_GRAPH if graph else 0
        flags |= capi.LB_PERSISTENT if persistent else 0
        flags |= capi.LB_AUTOTUNE if autotune else 0
        flags |= 0 if bulk else capi.LB_NO_BULK
        flags |= 0 if tensor_maps else capi.LB_NO_TENSOR_MAPS
        self.flags = flags
        self.precision = precision
        if allocator is None:
            self.h = capi.lb_create_batch([p.to_c() for p in self.lattices], flags)
        else:
            # the callbacks must outlive the context: they are kept on the object
            self._allocator = capi.torch_allocator() if allocator == "torch" else tuple(allocator)
            self.h = capi.lb_create_batch_with_allocator([p.to_c() for p in self.lattices], flags, *self._allocator)

    def close(self):
        if getattr(self, "h", None):
            capi.lb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- control
    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t handle, or None (own stream)."""
        handle = getattr(stream, "cuda_stream", stream)
        capi.lb_set_stream(self.h, handle or 0)

    def set_sampling(self, discard: int, every: int):
        capi.lb_set_sampling(self.h, discard, every)

    def set_tile(self, tile_x: int, rows_per_item: int):
        capi.lb_set_tile(self.h, tile_x, rows_per_item)

    def tile(self):
        return capi.lb_get_tile(self.h)

    def step(self, n: int = 1):
        capi.lb_step(self.h, n)

    def synchronize(self):
        capi.lb_synchronize(self.h)

    @property
    def time(self) -> int:
        return capi.lb_time(self.h)

    def reset_statistics(self):
        capi.lb_reset_statistics(self.h)

    def device_bytes(self) -> int:
        return capi.lb_device_bytes(self.h)

    def kernel_launches(self) -> int:
        return capi.lb_kernel_launches(self.h)

    # ---- results
    def shape(self, lattice: int = 0):
        return capi.lb_lattice_shape(self.h, lattice)

    def structure_factor(self, field: str = "c", lattice: int = 0, qz0_only: bool = False):
        Lx, Lz = self.shape(lattice)
        out = np.empty(Lx if qz0_only else (Lz, Lx), np.float64)
        n = capi.lb_structure_factor(self.h, lattice, FIELDS.get(field, field),
                                     capi.LB_SF_QX if qz0_only else capi.LB_SF_QXQZ, out)
        return out, n

    def profile(self, field: str = "p", lattice: int = 0):
        """Time-averaged z-profile (row means over x) of rho, c, ux, uz or p, and the sample count."""
        out = np.empty(self.shape(lattice)[1], np.float64)
        n = capi.lb_profile(self.h, lattice, FIELDS.get(field, field), out)
        return out, n

    def set_correlations(self, fields=("c", "ux"), modes=()):
        """Accumulate, from the next sample on, the real-space correlations of `fields` and their
        mixed correlations C(q_x, z, z') for the q_x mode indices `modes`."""
        mask = 0
        for f in fields:
            mask |= 1 << FIELDS.get(f, f)
        capi.lb_set_correlations(self.h, mask, list(modes))

    def correlation(self, field: str = "c", lattice: int = 0):
        """<dphi(x, z) dphi(x, z')> averaged over x and the samples, (Lz, Lz), and the count."""
        Lz = self.shape(lattice)[1]
        out = np.empty((Lz, Lz), np.float64)
        n = capi.lb_correlation(self.h, lattice, FIELDS.get(field, field), out)
        return out, n

    def mode_correlation(self, field: str = "c", mode_index: int = 0, lattice: int = 0):
        """C(q_x, z, z') of the mode_index-th requested mode, (Lz, Lz) complex, and the count."""
        Lz = self.shape(lattice)[1]
        out = np.empty((Lz, Lz, 2), np.float64)
        n = capi.lb_mode_correlation(self.h, lattice, FIELDS.get(field, field), mode_index, out)
        return out[..., 0] + 1j * out[..., 1], n

    def mean_pressure(self, lattice: int = 0):
        return capi.lb_mean_pressure(self.h, lattice)

    def mass(self, lattice: int = 0):
        return capi.lb_mass(self.h, lattice)

    def pressure_shift_gradient(self, steps: int, ckpt_every: int = 100, want_grad: bool = True):
        """(L, [dL/dG, dL/dlambda_s, dL/dlambda_d]) of the time-averaged mean-pressure shift from
        the rest state over `steps` steps (reverse sweep with checkpoints every `ckpt_every`)."""
        return capi.lb_pressure_shift_gradient(self.h, steps, min(ckpt_every, steps), want_grad)

    def pressure_shift_gradients(self, steps: int, ckpt_every: int = 100, want_grad: bool = True):
        """pressure_shift_gradient of every lattice of the batch in one sweep: (losses[n],
        grads[n, 3]); each lattice's results equal those of a context holding it alone."""
        return capi.lb_pressure_shift_gradient_batch(self.h, steps, min(ckpt_every, steps), len(self.lattices),
                                                     want_grad)

    def populations(self, lattice: int = 0) -> np.ndarray:
        Lx, Lz = self.shape(lattice)
        out = np.empty((2, 9, Lz, Lx), np.float64)
        capi.lb_get_populations(self.h, lattice, out)
        return out

    # ---- checkpoint / resume
    def save_checkpoint(self) -> np.ndarray:
        """The context's whole dynamic state (populations, step count, settings, accumulators) as
        bytes in host memory (a uint8 array); lb_load_checkpoint restores it."""
        buf = np.empty(capi.lb_checkpoint_bytes(self.h), np.uint8)
        capi.lb_save_checkpoint(self.h, buf)
        return buf

    def load_checkpoint(self, buf):
        """Resume from save_checkpoint's bytes (same lattices and result-affecting options)."""
        capi.lb_load_checkpoint(self.h, np.ascontiguousarray(buf, dtype=np.uint8))

    # ---- x-slab decomposition (one large lattice cut into windows of columns)
    def set_site_map(self, x0: int, Lx_global: int, lattice: int = 0):
        """Noise counters of column x of this lattice: those of column (x + x0) mod Lx_global of
        the undivided lattice (an x-slab window)."""
        capi.lb_set_site_map(self.h, lattice, x0, Lx_global)

    def export_columns(self, x_first: int, n_cols: int, out=None, lattice: int = 0):
        """Columns [x_first, x_first + n_cols) of the stored state as a torch tensor on the current
        device, [18][Lz][n_cols] in the storage type (ordered on the context's stream)."""
        import torch
        Lz = self.shape(lattice)[1]
        dt = torch.float32 if self.precision == "dev32" else torch.float64
        if out is None:
            out = torch.empty((18, Lz, n_cols), dtype=dt, device="cuda")
        if out.dtype != dt or out.numel() != 18 * Lz * n_cols or not out.is_contiguous():
            raise ValueError("export buffer: contiguous [18][Lz][n_cols] of the storage type")
        capi.lb_export_columns(self.h, lattice, x_first, n_cols, out.data_ptr())
        return out

    def import_columns(self, x_first: int, cols, lattice: int = 0):
        """Overwrite columns [x_first, x_first + n) of the stored state with a device tensor
        [18][Lz][n] in the storage type (ordered on the context's stream)."""
        import torch
        Lz = self.shape(lattice)[1]
        dt = torch.float32 if self.precision == "dev32" else torch.float64
        if cols.dtype != dt or cols.dim() != 3 or cols.shape[:2] != (18, Lz) or not cols.is_contiguous():
            raise ValueError("import buffer: contiguous [18][Lz][n] of the storage type")
        capi.lb_import_columns(self.h, lattice, x_first, cols.shape[2], cols.data_ptr())

    def set_populations(self, f: np.ndarray, lattice: int = 0):
        Lx, Lz = self.shape(lattice)
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(2, 9, Lz, Lx)
        capi.lb_set_populations(self.h, lattice, f)
