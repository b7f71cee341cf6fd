"""ctypes binding of the C interface in ``include/lb.h`` -- argument marshalling only.

Every function here has the name of the C call it wraps and raises :class:`LBError` on a
non-zero status.  The library must have been built (``paper_1808_05168_gb300.build``);
there is no fallback of any kind when it is missing.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

LB_OK = 0
LB_ERR_BAD_PARAM = -1
LB_ERR_OOM = -2
LB_ERR_CUDA = -3
LB_ERR_NONFINITE = -4
LB_ERR_TIMEOUT = -5
LB_ERR_SIZE = -6
LB_ERR_STATE = -7

LB_PREC_FP64 = 0x00
LB_PREC_DEV32 = 0x01
LB_NO_ASTAR = 0x02
LB_WALL_FIXED = 0x04
LB_NOISE_LOC = 0x08
LB_GRAPH = 0x10
LB_PERSISTENT = 0x20
LB_AUTOTUNE = 0x40
LB_NO_BULK = 0x80
LB_NO_TENSOR_MAPS = 0x100

LB_FIELD_RHO, LB_FIELD_C, LB_FIELD_UX, LB_FIELD_UZ, LB_FIELD_P = 0, 1, 2, 3, 4
LB_SF_QXQZ, LB_SF_QX = 0, 1

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "liblb_gb300.so")

# Every symbol declared in include/lb.h.
EXPORTS = ("lb_create", "lb_create_batch", "lb_create_batch_with_allocator", "lb_set_stream", "lb_set_sampling", "lb_set_tile", "lb_get_tile",
           "lb_step", "lb_synchronize", "lb_time", "lb_num_lattices", "lb_lattice_shape", "lb_structure_factor",
           "lb_profile", "lb_set_correlations", "lb_correlation", "lb_mode_correlation", "lb_mean_pressure", "lb_mass", "lb_get_populations", "lb_set_populations", "lb_reset_statistics",
           "lb_device_bytes", "lb_kernel_launches", "lb_error_string", "lb_destroy", "lb_debug_barrier",
           "lb_debug_box_muller", "lb_debug_schedule",
           "lb_power_spectrum", "lb_power_spectrum_noalloc", "lb_pressure_shift_gradient",
           "lb_pressure_shift_gradient_batch", "lb_set_site_map",
           "lb_export_columns", "lb_import_columns", "lb_debug_fma_rate", "lb_checkpoint_bytes",
           "lb_save_checkpoint", "lb_load_checkpoint")
LB_NOALLOC_MAX_POINTS = 1 << 18
LB_CORR_MAX_MODES = 16


class LBError(RuntimeError):
    def __init__(self, code: int, call: str):
        self.code = code
        msg = _lib.lb_error_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{call}: {msg} ({code})")


class lb_params(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int32), ("Lz", ctypes.c_int32), ("lambda_s", ctypes.c_double),
                ("lambda_d", ctypes.c_double), ("lambda_e", ctypes.c_double), ("lambda_q", ctypes.c_double),
                ("lambda_eps", ctypes.c_double), ("kT", ctypes.c_double), ("G", ctypes.c_double),
                ("grad_c0", ctypes.c_double), ("seed", ctypes.c_uint64), ("lattice_id", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


_lib = None
_lock = threading.Lock()


def load():
    """Load the compiled library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run `python -m paper_1808_05168_gb300.build`)")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i, i64, u64, d, sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double,
                                  ctypes.c_size_t)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        i64p = ctypes.POINTER(ctypes.c_int64)
        sig = {
            "lb_create": [ctypes.POINTER(vp), i, i, d, d, d, d, d, d, d, d, u64, i],
            "lb_create_batch": [ctypes.POINTER(vp), i, ctypes.POINTER(lb_params), i],
            "lb_create_batch_with_allocator": [ctypes.POINTER(vp), i, ctypes.POINTER(lb_params), i, LB_ALLOC_FN,
                                               LB_FREE_FN, vp],
            "lb_set_stream": [vp, vp],
            "lb_set_sampling": [vp, i64, i64],
            "lb_set_tile": [vp, i, i],
            "lb_get_tile": [vp, ip, ip],
            "lb_step": [vp, i64],
            "lb_synchronize": [vp],
            "lb_time": [vp, i64p],
            "lb_num_lattices": [vp, ip],
            "lb_lattice_shape": [vp, i, ip, ip],
            "lb_structure_factor": [vp, i, i, i, dp, sz, i64p],
            "lb_mean_pressure": [vp, i, dp, dp],
            "lb_profile": [vp, i, i, dp, sz, i64p],
            "lb_set_correlations": [vp, i, i, ip],
            "lb_correlation": [vp, i, i, dp, sz, i64p],
            "lb_mode_correlation": [vp, i, i, i, dp, sz, i64p],
            "lb_mass": [vp, i, dp],
            "lb_get_populations": [vp, i, dp, sz],
            "lb_set_populations": [vp, i, dp, sz],
            "lb_reset_statistics": [vp],
            "lb_device_bytes": [vp, ctypes.POINTER(sz)],
            "lb_kernel_launches": [vp, i64p],
            "lb_destroy": [vp],
            "lb_debug_barrier": [i, i, i],
            "lb_debug_box_muller": [i, ctypes.POINTER(ctypes.c_uint32), i64, dp],
            "lb_debug_schedule": [i, ip, ip, i, i, ip, i64, ip, ip, i64, i64p, i64p],
            "lb_power_spectrum": [vp, i, i, vp, vp],
            "lb_power_spectrum_noalloc": [vp, i, i, vp, vp],
            "lb_pressure_shift_gradient": [vp, i64, i64, dp, dp],
            "lb_pressure_shift_gradient_batch": [vp, i64, i64, dp, dp],
            "lb_set_site_map": [vp, i, i, i],
            "lb_export_columns": [vp, i, i, i, vp],
            "lb_import_columns": [vp, i, i, i, vp],
            "lb_debug_fma_rate": [i, dp],
            "lb_checkpoint_bytes": [vp, ctypes.POINTER(sz)],
            "lb_save_checkpoint": [vp, vp, sz],
            "lb_load_checkpoint": [vp, vp, sz],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = None if name == "lb_destroy" else ctypes.c_int
        lib.lb_error_string.argtypes = [ctypes.c_int]
        lib.lb_error_string.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _check(rc: int, call: str):
    if rc != LB_OK:
        raise LBError(rc, call)


def _dptr(a: np.ndarray):
    if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("expected a C-contiguous float64 array")
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a: np.ndarray):
    if a.dtype != np.int32 or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("expected a C-contiguous int32 array")
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def lb_create(Lx, Lz, lambda_s, lambda_d, lambda_e, lambda_q, lambda_eps, kT, G, grad_c0, seed, flags):
    lib = load()
    h = ctypes.c_void_p()
    _check(lib.lb_create(ctypes.byref(h), int(Lx), int(Lz), float(lambda_s), float(lambda_d), float(lambda_e),
                         float(lambda_q), float(lambda_eps), float(kT), float(G), float(grad_c0), int(seed),
                         int(flags)), "lb_create")
    return h


# Callback types of lb_create_batch_with_allocator: alloc(bytes, user) -> device pointer or NULL,
# free(ptr, user).
LB_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
LB_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


def torch_allocator(device=None):
    """(alloc, free) callbacks that take the context's device memory from torch's caching
    allocator on `device` (the current device by default).  Keep them alive as long as the
    context."""
    import torch

    dev = torch.cuda.current_device() if device is None else device

    def alloc(nbytes, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev)
        except Exception:
            return None

    def free(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)

    return LB_ALLOC_FN(alloc), LB_FREE_FN(free)


def lb_create_batch_with_allocator(params, flags, alloc_cb, free_cb):
    lib = load()
    arr = (lb_params * len(params))(*params)
    h = ctypes.c_void_p()
    _check(lib.lb_create_batch_with_allocator(ctypes.byref(h), len(params), arr, int(flags), alloc_cb, free_cb, None),
           "lb_create_batch_with_allocator")
    return h


def lb_create_batch(params, flags):
    lib = load()
    arr = (lb_params * len(params))(*params)
    h = ctypes.c_void_p()
    _check(lib.lb_create_batch(ctypes.byref(h), len(params), arr, int(flags)), "lb_create_batch")
    return h


def lb_set_stream(h, stream_handle):
    _check(load().lb_set_stream(h, ctypes.c_void_p(int(stream_handle) if stream_handle else 0)), "lb_set_stream")


def lb_set_sampling(h, discard, every):
    _check(load().lb_set_sampling(h, int(discard), int(every)), "lb_set_sampling")


def lb_set_tile(h, tile_x, rows_per_item):
    _check(load().lb_set_tile(h, int(tile_x), int(rows_per_item)), "lb_set_tile")


def lb_get_tile(h):
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(load().lb_get_tile(h, ctypes.byref(a), ctypes.byref(b)), "lb_get_tile")
    return a.value, b.value


def lb_step(h, n):
    _check(load().lb_step(h, int(n)), "lb_step")


def lb_synchronize(h):
    _check(load().lb_synchronize(h), "lb_synchronize")


def lb_time(h):
    t = ctypes.c_int64()
    _check(load().lb_time(h, ctypes.byref(t)), "lb_time")
    return t.value


def lb_num_lattices(h):
    n = ctypes.c_int()
    _check(load().lb_num_lattices(h, ctypes.byref(n)), "lb_num_lattices")
    return n.value


def lb_lattice_shape(h, lattice):
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(load().lb_lattice_shape(h, int(lattice), ctypes.byref(a), ctypes.byref(b)), "lb_lattice_shape")
    return a.value, b.value


def lb_structure_factor(h, lattice, field, mode, out: np.ndarray):
    n = ctypes.c_int64()
    _check(load().lb_structure_factor(h, int(lattice), int(field), int(mode), _dptr(out), out.size, ctypes.byref(n)),
           "lb_structure_factor")
    return n.value


def lb_profile(h, lattice, field, out: np.ndarray):
    n = ctypes.c_int64()
    _check(load().lb_profile(h, int(lattice), int(field), _dptr(out), out.size, ctypes.byref(n)), "lb_profile")
    return n.value


def lb_set_correlations(h, field_mask, modes=()):
    m = (ctypes.c_int * max(1, len(modes)))(*[int(k) for k in modes])
    _check(load().lb_set_correlations(h, int(field_mask), len(modes), m), "lb_set_correlations")


def lb_correlation(h, lattice, field, out: np.ndarray):
    n = ctypes.c_int64()
    _check(load().lb_correlation(h, int(lattice), int(field), _dptr(out), out.size, ctypes.byref(n)), "lb_correlation")
    return n.value


def lb_mode_correlation(h, lattice, field, mode_index, out: np.ndarray):
    n = ctypes.c_int64()
    _check(load().lb_mode_correlation(h, int(lattice), int(field), int(mode_index), _dptr(out), out.size,
                                      ctypes.byref(n)), "lb_mode_correlation")
    return n.value


def lb_mean_pressure(h, lattice):
    last, avg = ctypes.c_double(), ctypes.c_double()
    _check(load().lb_mean_pressure(h, int(lattice), ctypes.byref(last), ctypes.byref(avg)), "lb_mean_pressure")
    return last.value, avg.value


def lb_mass(h, lattice):
    out = np.empty(2, np.float64)
    _check(load().lb_mass(h, int(lattice), _dptr(out)), "lb_mass")
    return out


def lb_get_populations(h, lattice, out: np.ndarray):
    _check(load().lb_get_populations(h, int(lattice), _dptr(out), out.size), "lb_get_populations")


def lb_set_populations(h, lattice, src: np.ndarray):
    _check(load().lb_set_populations(h, int(lattice), _dptr(src), src.size), "lb_set_populations")


def lb_reset_statistics(h):
    _check(load().lb_reset_statistics(h), "lb_reset_statistics")


def lb_device_bytes(h):
    n = ctypes.c_size_t()
    _check(load().lb_device_bytes(h, ctypes.byref(n)), "lb_device_bytes")
    return n.value


def lb_kernel_launches(h):
    n = ctypes.c_int64()
    _check(load().lb_kernel_launches(h, ctypes.byref(n)), "lb_kernel_launches")
    return n.value


def lb_error_string(code):
    return load().lb_error_string(int(code)).decode()


def lb_destroy(h):
    if h:
        load().lb_destroy(h)


def lb_checkpoint_bytes(h) -> int:
    out = ctypes.c_size_t()
    _check(load().lb_checkpoint_bytes(h, ctypes.byref(out)), "lb_checkpoint_bytes")
    return int(out.value)


def lb_save_checkpoint(h, buf: np.ndarray):
    """buf: a C-contiguous uint8 array of exactly lb_checkpoint_bytes(h) bytes."""
    if buf.dtype != np.uint8 or not buf.flags["C_CONTIGUOUS"]:
        raise TypeError("expected a C-contiguous uint8 array")
    _check(load().lb_save_checkpoint(h, ctypes.c_void_p(buf.ctypes.data), buf.size), "lb_save_checkpoint")


def lb_load_checkpoint(h, buf: np.ndarray):
    if buf.dtype != np.uint8 or not buf.flags["C_CONTIGUOUS"]:
        raise TypeError("expected a C-contiguous uint8 array")
    _check(load().lb_load_checkpoint(h, ctypes.c_void_p(buf.ctypes.data), buf.size), "lb_load_checkpoint")


def lb_debug_fma_rate(precision) -> float:
    """Measured FMA rate of the current device in flop/s (LB_PREC_FP64: double, LB_PREC_DEV32: float)."""
    out = ctypes.c_double()
    _check(load().lb_debug_fma_rate(int(precision), ctypes.byref(out)), "lb_debug_fma_rate")
    return out.value


def lb_set_site_map(h, lattice, x0, Lx_global):
    _check(load().lb_set_site_map(h, int(lattice), int(x0), int(Lx_global)), "lb_set_site_map")


def lb_export_columns(h, lattice, x_first, n_cols, device_ptr):
    """device_ptr: device address of 18 * Lz * n_cols values of the storage type."""
    _check(load().lb_export_columns(h, int(lattice), int(x_first), int(n_cols), ctypes.c_void_p(int(device_ptr))),
           "lb_export_columns")


def lb_import_columns(h, lattice, x_first, n_cols, device_ptr):
    _check(load().lb_import_columns(h, int(lattice), int(x_first), int(n_cols), ctypes.c_void_p(int(device_ptr))),
           "lb_import_columns")


def lb_power_spectrum(field_ptr, Lx, Lz, out_ptr, stream_handle=0):
    """field_ptr, out_ptr: device addresses (e.g. torch tensor .data_ptr()) of Lx * Lz doubles."""
    _check(load().lb_power_spectrum(ctypes.c_void_p(int(field_ptr)), int(Lx), int(Lz), ctypes.c_void_p(int(out_ptr)),
                                    ctypes.c_void_p(int(stream_handle) if stream_handle else 0)), "lb_power_spectrum")


def lb_power_spectrum_noalloc(field_ptr, Lx, Lz, out_ptr, stream_handle=0):
    """As lb_power_spectrum, without any device allocation (Lx * Lz <= LB_NOALLOC_MAX_POINTS)."""
    _check(load().lb_power_spectrum_noalloc(ctypes.c_void_p(int(field_ptr)), int(Lx), int(Lz),
                                            ctypes.c_void_p(int(out_ptr)),
                                            ctypes.c_void_p(int(stream_handle) if stream_handle else 0)),
           "lb_power_spectrum_noalloc")


def lb_pressure_shift_gradient(h, steps, ckpt_every, want_grad=True):
    """(loss, grad[3] or None): see include/lb.h."""
    loss = ctypes.c_double()
    grad = np.zeros(3, np.float64)
    _check(load().lb_pressure_shift_gradient(h, int(steps), int(ckpt_every), _dptr(grad) if want_grad else None,
                                             ctypes.byref(loss)), "lb_pressure_shift_gradient")
    return loss.value, (grad if want_grad else None)


def lb_pressure_shift_gradient_batch(h, steps, ckpt_every, n_lattices, want_grad=True):
    """(losses[n], grads[n, 3] or None): see include/lb.h."""
    losses = np.zeros(int(n_lattices), np.float64)
    grads = np.zeros((int(n_lattices), 3), np.float64)
    _check(load().lb_pressure_shift_gradient_batch(h, int(steps), int(ckpt_every), _dptr(grads) if want_grad else None,
                                                   _dptr(losses)), "lb_pressure_shift_gradient_batch")
    return losses, (grads if want_grad else None)


def lb_debug_barrier(blocks, expected, limit_ms):
    return int(load().lb_debug_barrier(int(blocks), int(expected), int(limit_ms)))


def lb_debug_schedule(shapes, tile_x, rows):
    """(items [n, 4] = lattice, x0, z0, z1; off [n + 1]; nbr) of lattices shapes = [(Lx, Lz), ...]
    cut into tile_x x rows items: the work list and the persistent launch's dependency lists
    (host only; see include/lb.h)."""
    lx = np.ascontiguousarray([int(a) for a, _ in shapes], dtype=np.int32)
    lz = np.ascontiguousarray([int(b) for _, b in shapes], dtype=np.int32)
    ni, nn = ctypes.c_int64(), ctypes.c_int64()
    lib = load()
    rc = lib.lb_debug_schedule(len(shapes), _iptr(lx), _iptr(lz), int(tile_x), int(rows), None, 0, None, None, 0,
                               ctypes.byref(ni), ctypes.byref(nn))
    if rc not in (LB_OK, LB_ERR_SIZE):
        _check(rc, "lb_debug_schedule")
    items = np.zeros((ni.value, 4), np.int32)
    off = np.zeros(ni.value + 1, np.int32)
    nbr = np.zeros(max(nn.value, 1), np.int32)
    _check(lib.lb_debug_schedule(len(shapes), _iptr(lx), _iptr(lz), int(tile_x), int(rows), _iptr(items), ni.value,
                                 _iptr(off), _iptr(nbr), nn.value, ctypes.byref(ni), ctypes.byref(nn)),
           "lb_debug_schedule")
    return items, off, nbr[: nn.value]


def lb_debug_box_muller(precision, words):
    """Normals (2 per word pair) that the step kernels of `precision` form; see include/lb.h."""
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint32).reshape(-1))
    if w.size % 2:
        raise ValueError("words must hold pairs")
    out = np.empty(w.size, np.float64)
    _check(load().lb_debug_box_muller(int(precision), w.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                      w.size // 2, _dptr(out)), "lb_debug_box_muller")
    return out
