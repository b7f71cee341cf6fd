"""Gradient of the time-averaged mean-pressure shift (reverse sweep with checkpoints) against the
oracle's forward-mode dual-number gradient and against central differences of the library's own
loss on the same noise stream."""
import numpy as np
import pytest

import oracle
from paper_1808_05168_gb300 import LatticeParams, Simulation, capi, workloads

pytestmark = pytest.mark.gpu

SMALL = dict(Lx=16, Lz=8, kT=1e-3, G=0.5, grad_c0=0.05, lambda_s=1.2, lambda_d=0.9, lambda_e=1.0, seed=5)


def gpu_grad(p, steps, ckpt, precision="fp64", want_grad=True):
    with Simulation(p, precision=precision) as sim:
        return sim.pressure_shift_gradient(steps, ckpt, want_grad)


@pytest.mark.parametrize("prec,gtol,ltol", [("fp64", 1e-8, 1e-10), ("dev32", 3e-3, 1e-4)])
def test_adjoint_matches_oracle_dual_numbers(prec, gtol, ltol):
    p = LatticeParams(**SMALL)
    steps = 40
    loss, g = gpu_grad(p, steps, 7, prec)  # 6 segments, the last one shorter
    o_loss, o_g = oracle.pressure_shift_grad(p.Lx, p.Lz, steps, lambda_s=p.lambda_s, lambda_d=p.lambda_d,
                                             lambda_e=p.lambda_e, kT=p.kT, G=p.G, grad_c0=p.grad_c0, seed=p.seed)
    assert abs(loss - o_loss) <= ltol * abs(o_loss), (loss, o_loss)
    np.testing.assert_allclose(g, o_g, rtol=0, atol=gtol * np.max(np.abs(o_g)))


def test_checkpoint_interval_does_not_change_the_gradient():
    p = LatticeParams(**SMALL)
    _, g1 = gpu_grad(p, 30, 1)
    _, g2 = gpu_grad(p, 30, 30)
    _, g3 = gpu_grad(p, 30, 4)
    np.testing.assert_allclose(g1, g2, rtol=1e-13, atol=0)
    np.testing.assert_allclose(g1, g3, rtol=1e-13, atol=0)


def test_noiseless_shift_is_zero():
    """At kT = 0 both runs coincide: the loss vanishes and so does its gradient, up to the rounding
    of the two runs' sums (each run's dPbar/dG alone is about rho^A rho^B / 3 = 1/12)."""
    p = LatticeParams(**dict(SMALL, kT=0.0))
    loss, g = gpu_grad(p, 20, 5)
    assert loss == 0.0
    assert np.max(np.abs(g)) < 1e-13


def test_adjoint_matches_central_differences_full_size():
    """256 x 128, G = 0.5, wall-to-wall difference 0.5, kT = 1e-5, 2000 steps, checkpoints every
    100 steps; central differences with step 1e-4 on the same noise (FP64 storage: the FP32
    loss is not resolved to the 1e-10 that a step of 1e-4 needs)."""
    (p,) = workloads.c5()
    steps, h, rtol, prec = 2000, 1e-4, 1e-5, "fp64"
    loss, g = gpu_grad(p, steps, 100, prec)
    fd = []
    for key in ("G", "lambda_s", "lambda_d"):
        up = LatticeParams(**{**p.__dict__, key: getattr(p, key) + h})
        dn = LatticeParams(**{**p.__dict__, key: getattr(p, key) - h})
        lu, _ = gpu_grad(up, steps, 100, prec, want_grad=False)
        ld, _ = gpu_grad(dn, steps, 100, prec, want_grad=False)
        fd.append((lu - ld) / (2 * h))
    fd = np.array(fd)
    assert np.all(np.isfinite(g)) and abs(loss) > 0
    np.testing.assert_allclose(g, fd, rtol=0, atol=rtol * np.max(np.abs(fd)))


def test_fp32_gradient_follows_fp64_full_size():
    """The FP32-deviation run's gradient (its own trajectory, transposed in double precision)
    against the FP64 run's, on the 256 x 128, 2000-step configuration."""
    (p,) = workloads.c5()
    l64, g64 = gpu_grad(p, 2000, 100, "fp64")
    l32, g32 = gpu_grad(p, 2000, 100, "dev32")
    assert abs(l32 - l64) <= 5e-3 * abs(l64), (l32, l64)
    np.testing.assert_allclose(g32, g64, rtol=0, atol=2e-2 * np.max(np.abs(g64)))


@pytest.mark.parametrize("prec", ["fp64", "dev32"])
def test_gradient_does_not_depend_on_the_tile(prec):
    """The reverse sweep recomputes the forward states in buffers of its own; with tiles narrow
    enough for strips away from the x edges (staged by tensor copies in the forward run) it must
    give the default tile's states, hence its gradient, bit for bit (the loss sums per-item pressure
    partials, so its rounding follows the tile)."""
    p = LatticeParams(256, 16, kT=1e-4, G=0.5, grad_c0=0.02, seed=9)
    out = []
    for tile in (128, 64, 32):
        with Simulation(p, precision=prec) as sim:
            sim.set_tile(tile, 8)
            out.append(sim.pressure_shift_gradient(30, 7))
    for loss, g in out[1:]:
        assert abs(loss - out[0][0]) <= 1e-12 * abs(out[0][0])
        np.testing.assert_array_equal(g, out[0][1])


def test_autograd_function():
    import torch
    from paper_1808_05168_gb300.autograd import MeanPressureShift
    p = LatticeParams(**SMALL)
    G = torch.tensor(p.G, dtype=torch.float64, requires_grad=True)
    ls = torch.tensor(p.lambda_s, dtype=torch.float64, requires_grad=True)
    ld = torch.tensor(p.lambda_d, dtype=torch.float64, requires_grad=True)
    L = MeanPressureShift.apply(G, ls, ld, p, 25, 5)
    (2.0 * L).backward()
    loss, g = gpu_grad(p, 25, 5)
    assert float(L.detach()) == loss
    np.testing.assert_array_equal([G.grad.item(), ls.grad.item(), ld.grad.item()], 2.0 * g)


def test_batches_are_refused():
    with Simulation([LatticeParams(8, 4), LatticeParams(8, 4, lattice_id=1)]) as sim:
        with pytest.raises(capi.LBError) as e:
            sim.pressure_shift_gradient(10, 5)
        assert e.value.code == capi.LB_ERR_STATE


@pytest.mark.parametrize("prec", ["fp64", "dev32"])
def test_batch_gives_every_lattice_its_own_gradient(prec):
    """One sweep over a batch of different lattices (sizes, parameters, seeds, ids): each lattice's
    loss and gradient equal those of a context that holds it alone, bit for bit, and the oracle's
    dual numbers."""
    ps = [LatticeParams(**SMALL),
          LatticeParams(24, 6, kT=2e-3, G=0.3, grad_c0=0.04, lambda_s=1.1, lambda_d=1.3, lambda_e=0.9, seed=7,
                        lattice_id=1),
          LatticeParams(130, 12, kT=1e-3, G=0.6, grad_c0=-0.02, lambda_s=0.8, lambda_d=1.0, seed=5, lattice_id=2)]
    steps, ckpt = 30, 7
    with Simulation(ps, precision=prec) as sim:
        losses, grads = sim.pressure_shift_gradients(steps, ckpt)
    for i, p in enumerate(ps):
        with Simulation(p, precision=prec) as sim:
            loss, g = sim.pressure_shift_gradient(steps, ckpt)
        assert losses[i] == loss
        np.testing.assert_array_equal(grads[i], g)
        o_loss, o_g = oracle.pressure_shift_grad(p.Lx, p.Lz, steps, lambda_s=p.lambda_s, lambda_d=p.lambda_d,
                                                 lambda_e=p.lambda_e, kT=p.kT, G=p.G, grad_c0=p.grad_c0,
                                                 seed=p.seed, lattice_id=p.lattice_id)
        gtol = 1e-8 if prec == "fp64" else 3e-3
        np.testing.assert_allclose(g, o_g, rtol=0, atol=gtol * np.max(np.abs(o_g)))
    with Simulation(ps, precision=prec) as sim:
        losses2, none = sim.pressure_shift_gradients(steps, ckpt, want_grad=False)
    assert none is None
    np.testing.assert_array_equal(losses2, losses)


VARIANTS = {"no_astar": dict(astar=False), "wall_fixed": dict(wall_fixed=True), "noise_loc": dict(noise_loc=True),
            "all_three": dict(astar=False, wall_fixed=True, noise_loc=True)}


@pytest.mark.parametrize("prec,gtol,ltol", [("fp64", 1e-8, 1e-10), ("dev32", 3e-3, 1e-4)])
@pytest.mark.parametrize("variant", list(VARIANTS))
def test_adjoint_of_every_step_option_matches_oracle(variant, prec, gtol, ltol):
    """The options of the step (no a*, fixed wall composition in the ghosts of Sec. II.A, loc noise
    whose amplitudes follow the local densities) against the oracle's dual-number gradient of the
    same configuration."""
    opts = VARIANTS[variant]
    p = LatticeParams(**SMALL)
    with Simulation(p, precision=prec, **opts) as sim:
        loss, g = sim.pressure_shift_gradient(40, 7)
    o_loss, o_g = oracle.pressure_shift_grad(p.Lx, p.Lz, 40, lambda_s=p.lambda_s, lambda_d=p.lambda_d,
                                             lambda_e=p.lambda_e, kT=p.kT, G=p.G, grad_c0=p.grad_c0, seed=p.seed,
                                             **opts)
    assert abs(loss - o_loss) <= ltol * abs(o_loss), (loss, o_loss)
    np.testing.assert_allclose(g, o_g, rtol=0, atol=gtol * np.max(np.abs(o_g)))


def test_autograd_function_with_step_options():
    import torch
    from paper_1808_05168_gb300.autograd import MeanPressureShift
    p = LatticeParams(**SMALL)
    opts = VARIANTS["all_three"]
    G = torch.tensor(p.G, dtype=torch.float64, requires_grad=True)
    ls = torch.tensor(p.lambda_s, dtype=torch.float64, requires_grad=True)
    ld = torch.tensor(p.lambda_d, dtype=torch.float64, requires_grad=True)
    L = MeanPressureShift.apply(G, ls, ld, p, 25, 5, "fp64", opts)
    L.backward()
    with Simulation(p, precision="fp64", **opts) as sim:
        loss, g = sim.pressure_shift_gradient(25, 5)
    assert float(L.detach()) == loss
    np.testing.assert_array_equal([G.grad.item(), ls.grad.item(), ld.grad.item()], g)
