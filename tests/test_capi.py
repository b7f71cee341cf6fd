"""The C interface without a GPU: the library builds, loads, exports every symbol that
include/lb.h declares, and rejects bad arguments before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1808_05168_gb300 import build, capi
    build.build()
    return capi.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "lb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z_]+)\s*\(", src)))


def test_header_and_binding_agree():
    from paper_1808_05168_gb300 import capi
    assert _declared() == sorted(capi.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_error_strings(lib):
    from paper_1808_05168_gb300 import capi
    assert capi.lb_error_string(0) == "ok"
    for code in range(-7, 0):
        assert capi.lb_error_string(code) not in ("ok", "unknown error")


@pytest.mark.parametrize("kw", [
    dict(Lx=0), dict(Lz=1), dict(lambda_s=0.0), dict(lambda_d=2.0), dict(lambda_eps=-1.0), dict(kT=-1e-5),
    dict(G=-0.1), dict(grad_c0=0.05), dict(flags=0x1000), dict(lambda_q=float("nan")),
])
def test_bad_parameters_are_rejected_without_a_device(lib, kw):
    from paper_1808_05168_gb300 import capi
    args = dict(Lx=16, Lz=20, lambda_s=1.0, lambda_d=0.8, lambda_e=1.0, lambda_q=1.0, lambda_eps=1.0, kT=1e-5,
                G=0.5, grad_c0=0.01, seed=1, flags=0)
    args.update(kw)
    h = ctypes.c_void_p(123)
    rc = lib.lb_create(ctypes.byref(h), args["Lx"], args["Lz"], args["lambda_s"], args["lambda_d"], args["lambda_e"],
                       args["lambda_q"], args["lambda_eps"], args["kT"], args["G"], args["grad_c0"], args["seed"],
                       args["flags"])
    assert rc == capi.LB_ERR_BAD_PARAM
    assert not h.value


def test_null_context_calls_fail_cleanly(lib):
    from paper_1808_05168_gb300 import capi
    assert lib.lb_step(None, 1) == capi.LB_ERR_BAD_PARAM
    assert lib.lb_synchronize(None) == capi.LB_ERR_BAD_PARAM
    assert lib.lb_mass(None, 0, None) == capi.LB_ERR_BAD_PARAM
    assert lib.lb_debug_barrier(0, 1, 10) == capi.LB_ERR_BAD_PARAM
    assert lib.lb_profile(None, 0, capi.LB_FIELD_P, None, 0, None) == capi.LB_ERR_BAD_PARAM
    h = ctypes.c_void_p()
    p = capi.lb_params(8, 8, 1.0, 0.8, 1.0, 1.0, 1.0, 0.0, 0.0, 0.0, 1, 0, 0)
    assert lib.lb_create_batch_with_allocator(ctypes.byref(h), 1, (capi.lb_params * 1)(p), 0, capi.LB_ALLOC_FN(),
                                              capi.LB_FREE_FN(), None) == capi.LB_ERR_BAD_PARAM
    assert not h.value
    assert lib.lb_debug_box_muller(7, None, 1, None) == capi.LB_ERR_BAD_PARAM
    assert lib.lb_debug_box_muller(capi.LB_PREC_DEV32, None, -1, None) == capi.LB_ERR_BAD_PARAM
    assert lib.lb_debug_box_muller(capi.LB_PREC_DEV32, None, 1, None) == capi.LB_ERR_BAD_PARAM
    lib.lb_destroy(None)


def test_batch_rejects_reserved_field(lib):
    from paper_1808_05168_gb300 import capi
    p = capi.lb_params(8, 8, 1.0, 0.8, 1.0, 1.0, 1.0, 0.0, 0.0, 0.0, 1, 0, 7)
    h = ctypes.c_void_p()
    assert lib.lb_create_batch(ctypes.byref(h), 1, (capi.lb_params * 1)(p), 0) == capi.LB_ERR_BAD_PARAM
    assert lib.lb_create_batch(ctypes.byref(h), 0, None, 0) == capi.LB_ERR_BAD_PARAM


@pytest.mark.parametrize("fail_at", [0, 1, 3, 7])
def test_allocation_failure_is_reported_and_cleaned_up(lib, fail_at):
    """An allocator that refuses its (fail_at + 1)-th request (host-side fault injection, no GPU
    needed: the context's first allocations precede any device call): lb_create_batch_with_allocator
    returns LB_ERR_OOM, leaves *out NULL, and hands every pointer it did get back to free_fn, once."""
    from paper_1808_05168_gb300 import capi
    given, freed = [], []

    def alloc(nbytes, user):
        if len(given) == fail_at:
            return None
        given.append(0x10000 * (len(given) + 1))  # never dereferenced on the host
        return given[-1]

    def free(ptr, user):
        freed.append(ptr)

    a, f = capi.LB_ALLOC_FN(alloc), capi.LB_FREE_FN(free)
    p = capi.lb_params(64, 16, 1.0, 0.8, 1.0, 1.0, 1.0, 1e-5, 0.5, 0.01, 1, 0, 0)
    h = ctypes.c_void_p()
    rc = lib.lb_create_batch_with_allocator(ctypes.byref(h), 1, (capi.lb_params * 1)(p), capi.LB_PREC_DEV32, a, f,
                                            None)
    assert rc == capi.LB_ERR_OOM
    assert not h.value
    assert len(given) == fail_at and sorted(freed) == sorted(given)
