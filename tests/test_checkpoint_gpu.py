"""Checkpoint and resume through the C interface: a run stopped at step 80, saved, and resumed in
a fresh context reproduces the uninterrupted run bit for bit -- populations, structure factors
of every field, profiles, correlations, mean pressure, mass and the step count (which keys the
noise) -- for both precisions, for a batch of two lattices with sampling and correlations on, also
when the resumed context uses other launch options (CUDA graphs and the persistent launch)."""
import numpy as np
import pytest

from paper_1808_05168_gb300 import LatticeParams, Simulation, capi

pytestmark = pytest.mark.gpu

PS = [LatticeParams(64, 16, kT=1e-4, G=0.5, grad_c0=0.3 / 16, seed=31, lattice_id=0),
      LatticeParams(32, 8, lambda_s=1.3, kT=2e-4, G=0.3, grad_c0=-0.2 / 8, seed=32, lattice_id=1)]
FIELDS = ("rho", "c", "ux", "uz")


def outputs(sim):
    out = {"t": sim.time}
    for i in range(len(PS)):
        out[i] = dict(f=sim.populations(i), S={f: sim.structure_factor(f, lattice=i) for f in FIELDS},
                      prof={f: sim.profile(f, lattice=i) for f in FIELDS + ("p",)},
                      R={f: sim.correlation(f, lattice=i) for f in ("c", "ux")},
                      C=sim.mode_correlation("c", 1, lattice=i), P=sim.mean_pressure(i), m=sim.mass(i))
    return out


def assert_same(a, b, exact_pressure=True):
    assert a["t"] == b["t"]
    for i in range(len(PS)):
        x, y = a[i], b[i]
        np.testing.assert_array_equal(x["f"], y["f"])
        for f in FIELDS:
            np.testing.assert_array_equal(x["S"][f][0], y["S"][f][0])
            assert x["S"][f][1] == y["S"][f][1]
        for f in FIELDS + ("p",):
            np.testing.assert_array_equal(x["prof"][f][0], y["prof"][f][0])
        for f in ("c", "ux"):
            np.testing.assert_array_equal(x["R"][f][0], y["R"][f][0])
            assert x["R"][f][1] == y["R"][f][1]
        np.testing.assert_array_equal(x["C"][0], y["C"][0])
        np.testing.assert_array_equal(x["m"], y["m"])
        if exact_pressure:
            assert x["P"] == y["P"]
        else:  # another tile groups the double-precision pressure sums differently
            np.testing.assert_allclose(x["P"], y["P"], rtol=1e-14)


@pytest.mark.parametrize("prec", ["fp64", "dev32"])
def test_resumed_run_equals_the_uninterrupted_one(prec):
    with Simulation(PS, precision=prec) as sim:
        sim.set_sampling(10, 7)
        sim.set_correlations(("c", "ux"), [1, 3])
        sim.step(80)
        ck = sim.save_checkpoint()
        assert ck.size == capi.lb_checkpoint_bytes(sim.h)
        sim.step(70)
        want = outputs(sim)
    for kw in (dict(), dict(graph=True, persistent=True)):
        with Simulation(PS, precision=prec, **kw) as sim:
            sim.load_checkpoint(ck)
            assert sim.time == 80
            sim.step(70)
            assert_same(outputs(sim), want, exact_pressure=not kw)


def test_checkpoints_are_checked():
    with Simulation(PS, precision="dev32") as sim:
        sim.set_sampling(0, 5)
        sim.step(12)
        ck = sim.save_checkpoint()
        with pytest.raises(capi.LBError) as e:  # wrong size
            capi.lb_save_checkpoint(sim.h, np.empty(ck.size - 1, np.uint8))
        assert e.value.code == capi.LB_ERR_SIZE
    bad = ck.copy()
    bad[:8] = 0  # not a checkpoint
    other = [PS[0], LatticeParams(32, 8, lambda_s=1.3, kT=2e-4, G=0.3, grad_c0=-0.2 / 8, seed=33, lattice_id=1)]
    with Simulation(PS, precision="dev32") as sim:
        with pytest.raises(capi.LBError) as e:
            sim.load_checkpoint(bad)
        assert e.value.code == capi.LB_ERR_BAD_PARAM
        with pytest.raises(capi.LBError) as e:
            sim.load_checkpoint(ck[:-8])
        assert e.value.code == capi.LB_ERR_BAD_PARAM
    for lattices, prec in ((other, "dev32"), (PS, "fp64"), (PS[:1], "dev32")):
        with Simulation(lattices, precision=prec) as sim:
            with pytest.raises(capi.LBError) as e:
                sim.load_checkpoint(ck)
            assert e.value.code == capi.LB_ERR_STATE


def test_loading_replaces_earlier_statistics():
    """A context that has sampled before takes the checkpoint's statistics, not its own: a checkpoint
    saved before any sampling, loaded into a context with accumulated spectra, continues exactly as
    the saving context does."""
    with Simulation(PS, precision="dev32") as sim:
        sim.step(30)
        ck = sim.save_checkpoint()
        sim.set_sampling(0, 5)
        sim.step(20)
        want = outputs_spectra(sim)
    with Simulation(PS, precision="dev32") as sim:
        sim.set_sampling(0, 5)
        sim.step(20)
        assert sim.structure_factor("c")[1] == 4
        sim.load_checkpoint(ck)
        assert sim.time == 30 and sim.structure_factor("c")[1] == 0
        assert np.all(sim.structure_factor("c")[0] == 0)
        sim.set_sampling(0, 5)
        sim.step(20)
        got = outputs_spectra(sim)
    for a, b in zip(got, want):
        np.testing.assert_array_equal(a, b)


def outputs_spectra(sim):
    return [sim.populations(0), sim.structure_factor("c")[0], sim.structure_factor("uz", lattice=1)[0],
            np.array(sim.mean_pressure(1)), sim.profile("p")[0]]
