"""Parity of the CUDA path (through the C interface) with the oracle, element by element, on
the same seeded inputs and noise stream.

Tolerances: FP64 storage -- 1e-12 relative per population after up to 1000 steps; FP32
deviation storage -- absolute error at most 1e-5 of the largest deviation from the
background w_l rho_bar c^S_0(z); averaged diagnostics as stated per test.
"""
import numpy as np
import pytest

import oracle
from paper_1808_05168_gb300 import LatticeParams, Simulation, capi

pytestmark = pytest.mark.gpu

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1808_05168_gb300 import build
    build.build()
    oracle.build()


def background(Lx, Lz, grad_c0):
    z = np.arange(Lz) + 0.5 - Lz / 2
    c0 = 0.5 + z * grad_c0
    b = np.empty((2, 9, Lz, Lx))
    for l in range(9):
        b[0, l] = (W[l] * c0)[:, None]
        b[1, l] = (W[l] * (1 - c0))[:, None]
    return b


def oracle_of(p: LatticeParams, **flags):
    return oracle.OracleLattice(p.Lx, p.Lz, lambda_s=p.lambda_s, lambda_d=p.lambda_d, lambda_e=p.lambda_e,
                                lambda_q=p.lambda_q, lambda_eps=p.lambda_eps, kT=p.kT, G=p.G, grad_c0=p.grad_c0,
                                seed=p.seed, lattice_id=p.lattice_id, **flags)


def assert_fp64_parity(got, want, rtol=1e-12):
    err = np.abs(got - want) / np.maximum(np.abs(want), 1e-300)
    assert np.max(err) <= rtol, f"max relative error {np.max(err):.3e}"


def assert_dev32_parity(got, want, b, tol=1e-5):
    dev = want - b
    scale = np.max(np.abs(dev))
    err = np.max(np.abs(got - want))
    assert err <= tol * scale, f"max abs error {err:.3e} vs deviation scale {scale:.3e}"


C1 = LatticeParams(64, 32, lambda_s=1.0, lambda_d=0.8, kT=1e-5, G=0.0, grad_c0=0.5 / 32, seed=1)


def test_fp64_ideal_mixture_1000_steps():
    """64 x 32 ideal mixture with a wall-to-wall concentration difference of 0.5."""
    with Simulation(C1, precision="fp64") as sim:
        sim.step(1000)
        got = sim.populations()
    o = oracle_of(C1)
    o.step(1000)
    assert_fp64_parity(got, o.populations())


NI = LatticeParams(100, 20, lambda_s=1.3, lambda_d=0.9, lambda_e=1.1, lambda_q=1.2, lambda_eps=1.4, kT=1e-5, G=0.5,
                   grad_c0=0.4 / 20, seed=7)


@pytest.mark.parametrize("tile", [(64, 7), (128, 20), (32, 3)])
def test_fp64_nonideal_ragged_tiles(tile):
    """Non-ideal mixture on a ragged lattice (Lx not a tile multiple, Lz not a row multiple)."""
    with Simulation(NI, precision="fp64") as sim:
        sim.set_tile(*tile)
        sim.step(300)
        got = sim.populations()
    o = oracle_of(NI)
    o.step(300)
    assert_fp64_parity(got, o.populations())


@pytest.mark.parametrize("prec", ["fp64", "dev32"])
@pytest.mark.parametrize("variant", ["no_astar", "wall_fixed", "noise_loc", "all_three"])
def test_variants(variant, prec):
    """The method's variants, each a kernel instantiation of its own, in both precisions, 1000
    steps: a* off (footnote to Eq. ne-acc), fixed wall composition of the non-ideal force's ghost
    rows (Sec. II.A), noise variances from the local densities (loc, Sec. III.B), and all three
    together; G > 0 and rates != 1 so that every term is exercised."""
    p = LatticeParams(40, 12, lambda_s=1.2, lambda_d=1.1, kT=1e-4, G=0.6, grad_c0=0.3 / 12, seed=3)
    kw = {"no_astar": dict(astar=False), "wall_fixed": dict(wall_fixed=True), "noise_loc": dict(noise_loc=True),
          "all_three": dict(astar=False, wall_fixed=True, noise_loc=True)}
    with Simulation(p, precision=prec, **kw[variant]) as sim:
        sim.step(1000)
        got = sim.populations()
    o = oracle_of(p, **kw[variant])
    o.step(1000)
    if prec == "fp64":
        assert_fp64_parity(got, o.populations())
    else:
        assert_dev32_parity(got, o.populations(), background(p.Lx, p.Lz, p.grad_c0))


C2_SMALL = LatticeParams(64, 32, lambda_s=1.0, lambda_d=0.8, kT=1e-5, G=0.5, grad_c0=0.5 / 32, seed=2)


@pytest.mark.parametrize("p", [C1, C2_SMALL], ids=["ideal", "nonideal"])
def test_dev32_1000_steps(p):
    """FP32 deviations from the background against the FP64 oracle after 1000 steps."""
    with Simulation(p, precision="dev32") as sim:
        sim.step(1000)
        got = sim.populations()
    o = oracle_of(p)
    o.step(1000)
    assert_dev32_parity(got, o.populations(), background(p.Lx, p.Lz, p.grad_c0))


def test_batch_of_heterogeneous_lattices():
    """Three lattices of different sizes and parameters in one launch per step; each keeps its
    own noise stream (lattice_id is a Philox counter word)."""
    ps = [LatticeParams(64, 16, kT=1e-5, G=0.0, grad_c0=0.01, seed=1, lattice_id=0),
          LatticeParams(32, 8, lambda_s=1.4, kT=1e-4, G=0.5, grad_c0=0.02, seed=2, lattice_id=3),
          LatticeParams(100, 10, lambda_d=1.2, kT=1e-5, G=0.3, grad_c0=-0.03, seed=2, lattice_id=5)]
    for prec in ("fp64", "dev32"):
        with Simulation(ps, precision=prec) as sim:
            sim.step(200)
            got = [sim.populations(i) for i in range(3)]
        for i, p in enumerate(ps):
            o = oracle_of(p)
            o.step(200)
            if prec == "fp64":
                assert_fp64_parity(got[i], o.populations())
            else:
                assert_dev32_parity(got[i], o.populations(), background(p.Lx, p.Lz, p.grad_c0))


@pytest.mark.parametrize("prec", ["fp64", "dev32"])
def test_sampled_structure_factors_and_pressure(prec):
    """Appendix A structure factors (all four fields, full q grid) and the Sec. III.C mean
    pressure, sampled on the pre-collision state every 5 steps after 10."""
    p = LatticeParams(32, 16, lambda_s=1.1, lambda_d=0.9, kT=1e-4, G=0.5, grad_c0=0.3 / 16, seed=4)
    with Simulation(p, precision=prec) as sim:
        sim.set_sampling(10, 5)
        sim.step(101)
        S = {f: sim.structure_factor(f) for f in ("rho", "c", "ux", "uz")}
        Sqx = sim.structure_factor("c", qz0_only=True)
        last, avg = sim.mean_pressure()
    o = oracle_of(p)
    o.set_sampling(10, 5)
    o.step(101)
    for f in S:
        want, n = o.structure_factor(f)
        got, ng = S[f]
        assert n == ng == 19
        if prec == "fp64":
            np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-12 * want.max())
        else:
            assert np.max(np.abs(got - want)) <= 2e-3 * want.mean(), f
    np.testing.assert_array_equal(Sqx[0], S["c"][0][0])
    olast, oavg, _ = o.mean_pressure()
    tol = 1e-12 if prec == "fp64" else 1e-7
    assert abs(last - olast) <= tol * abs(olast)
    assert abs(avg - oavg) <= tol * abs(oavg)


@pytest.mark.parametrize("prec", ["fp64", "dev32"])
def test_profiles_of_a_batch(prec):
    """Sec. III.C z-profiles of rho, c, U and the pressure (time averages of row means on the
    sampled pre-collision state) for each lattice of a heterogeneous batch, against the oracle.
    FP32 deviations: the row means of the deviations from the background agree to 1e-5 of the
    largest such deviation (plus 1e-12 absolute), the bar of the populations."""
    ps = [LatticeParams(32, 16, kT=1e-4, G=0.5, grad_c0=0.3 / 16, seed=4, lattice_id=0),
          LatticeParams(64, 8, kT=2e-4, G=0.3, grad_c0=-0.2 / 8, seed=4, lattice_id=1)]
    with Simulation(ps, precision=prec) as sim:
        sim.set_sampling(10, 4)
        sim.step(83)
        got = [{f: sim.profile(f, lattice=i) for f in ("rho", "c", "ux", "uz", "p")} for i in range(2)]
    for i, p in enumerate(ps):
        o = oracle_of(p)
        o.set_sampling(10, 4)
        o.step(83)
        z = np.arange(p.Lz) + 0.5 - p.Lz / 2
        bg = {"rho": 1.0, "c": 0.5 + z * p.grad_c0, "ux": 0.0, "uz": 0.0, "p": None}
        for f, (g, n) in got[i].items():
            want, no = o.profile(f)
            assert n == no == 19
            if prec == "fp64":
                np.testing.assert_allclose(g, want, rtol=1e-12, atol=1e-15)
            else:
                b = bg[f] if bg[f] is not None else want.mean()
                scale = np.max(np.abs(want - b))
                assert np.max(np.abs(g - want)) <= 1e-5 * scale + 1e-12, (i, f, np.max(np.abs(g - want)), scale)
    with Simulation(ps, precision=prec) as sim:
        assert np.all(sim.profile("p", lattice=1)[0] == 0) and sim.profile("p", lattice=1)[1] == 0
        with pytest.raises(capi.LBError):
            capi.lb_profile(sim.h, 0, capi.LB_FIELD_P, np.empty(15))


@pytest.mark.parametrize("prec", ["fp64", "dev32"])
def test_tensor_copies_of_link_runs_match_1d_copies_and_oracle(prec):
    """Strips away from the periodic x edges are staged by 3-d tensor copies of runs of links
    (8-byte (A, B) pair elements, FP32 state); the result is bit-identical to 1-d copies per link
    row, for every tile width that uses them, per-step and persistent launches, and matches the
    oracle."""
    p = LatticeParams(512, 32, kT=1e-5, G=0.5, grad_c0=0.4 / 32, seed=13)
    o = oracle_of(p)
    o.set_sampling(0, 5)
    o.step(20)
    want = o.populations()
    base = None
    for tile in [(128, 7), (64, 32), (32, 5)]:
        for kw in (dict(tensor_maps=False), dict(), dict(persistent=True), dict(persistent=True, graph=True)):
            with Simulation(p, precision=prec, **kw) as sim:
                sim.set_tile(*tile)
                sim.set_sampling(0, 5)
                sim.step(20)
                r = (sim.populations(), sim.structure_factor("c")[0], sim.mean_pressure())
            if base is None:
                base = r
                if prec == "fp64":
                    assert_fp64_parity(r[0], want)
                else:
                    assert_dev32_parity(r[0], want, background(p.Lx, p.Lz, p.grad_c0))
            else:
                np.testing.assert_array_equal(r[0], base[0])
                np.testing.assert_array_equal(r[1], base[1])
                np.testing.assert_allclose(r[2], base[2], rtol=1e-14)


def test_tensor_copies_in_a_mixed_batch():
    """A batch of lattices of different widths (tensor maps per lattice and state buffer):
    persistent launches with tensor copies equal 1-d copies bit for bit, and every lattice
    matches its oracle."""
    ps = [LatticeParams(1024, 16, kT=1e-5, G=0.5, grad_c0=0.3 / 16, seed=21, lattice_id=0),
          LatticeParams(256, 32, kT=1e-5, G=0.5, grad_c0=0.5 / 32, seed=22, lattice_id=1),
          LatticeParams(512, 8, kT=1e-5, G=0.3, grad_c0=0.1 / 8, seed=23, lattice_id=2)]
    res = []
    for tm in (True, False):
        with Simulation(ps, precision="fp64", persistent=True, graph=True, tensor_maps=tm) as sim:
            sim.set_tile(64, 16)
            sim.step(11)
            res.append([sim.populations(i) for i in range(len(ps))])
    for a, b in zip(res[0], res[1]):
        np.testing.assert_array_equal(a, b)
    for i, p in enumerate(ps):
        o = oracle_of(p)
        o.step(11)
        assert_fp64_parity(res[0][i], o.populations())


@pytest.mark.parametrize("prec", ["fp64", "dev32"])
def test_launch_modes_and_tiles_are_bit_identical(prec):
    """Direct launches, CUDA graphs, the persistent cooperative launch and every tile shape
    compute each site identically."""
    p = LatticeParams(128, 32, kT=1e-5, G=0.5, grad_c0=0.4 / 32, seed=9)
    results = []
    configs = [dict(), dict(graph=True), dict(persistent=True), dict(graph=True, persistent=True), dict(bulk=False),
               dict(bulk=False, persistent=True)]
    for kw in configs:
        with Simulation(p, precision=prec, **kw) as sim:
            sim.set_sampling(3, 7)
            sim.step(70)
            sim.step(33)
            results.append((sim.populations(), sim.mean_pressure(), sim.structure_factor("c")[0],
                            sim.profile("p")[0]))
    for tile in [(32, 5), (256, 32), (64, 1)]:
        with Simulation(p, precision=prec) as sim:
            sim.set_tile(*tile)
            sim.set_sampling(3, 7)
            sim.step(103)
            results.append((sim.populations(), sim.mean_pressure(), sim.structure_factor("c")[0],
                            sim.profile("p")[0]))
    for i, r in enumerate(results[1:], start=1):
        np.testing.assert_array_equal(r[0], results[0][0])
        np.testing.assert_array_equal(r[2], results[0][2])
        np.testing.assert_array_equal(r[3], results[0][3])
        if i < len(configs):
            assert r[1] == results[0][1]
        else:  # another tile groups the double-precision pressure sums differently
            np.testing.assert_allclose(r[1], results[0][1], rtol=1e-14)


@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-13), ("dev32", 2e-8)])
def test_mass_is_conserved(prec, rtol):
    """Per-species mass (Sec. II.A).  FP64 storage conserves it to round-off; FP32 deviation
    storage rounds every post-collision population, a random walk of about 1e-9 relative over
    500 steps at kT = 1e-4 (the sums themselves are taken in double precision)."""
    p = LatticeParams(64, 32, kT=1e-4, G=0.5, grad_c0=0.01, seed=5)
    with Simulation(p, precision=prec) as sim:
        m0 = sim.mass()
        np.testing.assert_allclose(m0, [1024, 1024], rtol=1e-14)
        sim.step(500)
        np.testing.assert_allclose(sim.mass(), m0, rtol=rtol)


@pytest.mark.parametrize("prec", ["fp64", "dev32"])
def test_set_get_round_trip(prec):
    p = LatticeParams(33, 7, G=0.2, grad_c0=0.05)
    f = background(33, 7, 0.05) * (1 + 0.01 * np.random.default_rng(0).standard_normal((2, 9, 7, 33)))
    with Simulation(p, precision=prec) as sim:
        sim.set_populations(f)
        g = sim.populations()
    if prec == "fp64":
        np.testing.assert_array_equal(g, f)
    else:
        np.testing.assert_allclose(g, f, rtol=0, atol=1e-9)


@pytest.mark.parametrize("prec", ["fp64", "dev32"])
def test_multi_strip_lattice_wraps_periodically(prec):
    """Three column strips of 128 (bulk copies with the periodic wrap at both lattice edges and
    an interior strip), against the oracle."""
    p = LatticeParams(384, 12, lambda_s=1.2, lambda_d=0.9, kT=1e-4, G=0.4, grad_c0=0.3 / 12, seed=21)
    with Simulation(p, precision=prec) as sim:
        sim.set_tile(128, 5)
        sim.step(150)
        got = sim.populations()
    o = oracle_of(p)
    o.step(150)
    if prec == "fp64":
        assert_fp64_parity(got, o.populations())
    else:
        assert_dev32_parity(got, o.populations(), background(p.Lx, p.Lz, p.grad_c0))


def test_step_from_arbitrary_state():
    """One step from a random perturbed state (not reachable from rest) matches the oracle."""
    p = LatticeParams(48, 10, lambda_s=0.7, lambda_d=1.6, kT=1e-3, G=0.8, grad_c0=0.02, seed=11)
    f = background(48, 10, 0.02) * (1 + 0.05 * np.random.default_rng(1).standard_normal((2, 9, 10, 48)))
    with Simulation(p, precision="fp64") as sim:
        sim.set_populations(f)
        sim.step(3)
        got = sim.populations()
    o = oracle_of(p)
    o.set_populations(f)
    o.step(3)
    assert_fp64_parity(got, o.populations())


def test_bounded_grid_barrier_gives_up():
    """The grid barrier of the persistent launch waits a bounded time and reports a timeout
    (a barrier expecting more blocks than were launched), without hanging the device."""
    assert capi.lb_debug_barrier(2, 2, 500) == capi.LB_OK
    assert capi.lb_debug_barrier(2, 3, 300) == capi.LB_ERR_TIMEOUT
    assert capi.lb_debug_barrier(4, 4, 500) == capi.LB_OK


def test_errors_on_device():
    with Simulation(LatticeParams(30, 8), precision="fp64") as sim:
        with pytest.raises(capi.LBError) as e:
            sim.set_sampling(0, 1)  # Lx not a power of two
        assert e.value.code == capi.LB_ERR_BAD_PARAM
        with pytest.raises(capi.LBError) as e:
            capi.lb_get_populations(sim.h, 0, np.empty(5))
        assert e.value.code == capi.LB_ERR_SIZE
        with pytest.raises(capi.LBError):
            sim.populations(1)


def test_measured_fma_rates_are_plausible():
    """lb_debug_fma_rate, the ceiling of the FP64 path: GB300's FP64 FMA rate is about 1.25
    TFLOP/s and its FP32 one about 80 TFLOP/s (152 SMs, 128 lanes, about 2 GHz)."""
    f64 = capi.lb_debug_fma_rate(capi.LB_PREC_FP64)
    f32 = capi.lb_debug_fma_rate(capi.LB_PREC_DEV32)
    assert 0.5e12 < f64 < 2.5e12, f64
    assert 20e12 < f32 < 120e12, f32
    with pytest.raises(capi.LBError):
        capi.lb_debug_fma_rate(7)


def test_box_muller_normals_of_both_precisions():
    """The normals the step kernels draw, against the oracle's FP64 Box-Muller: random word
    pairs, every u1 of the band below 1 where the FP32 radius switches to its series, and the
    smallest u1 (the largest radii).  FP64 agrees to rounding; FP32 within 3e-6 absolute."""
    rng = np.random.default_rng(11)
    m = 1 << 18
    a = np.concatenate([rng.integers(0, 1 << 32, m, dtype=np.uint64),
                        np.arange((1 << 23) - (1 << 18), 1 << 23, dtype=np.uint64),  # v = 1 - u1 < 2^-5
                        np.arange(0, 1 << 14, dtype=np.uint64)])                       # u1 < 2^-9
    b = rng.integers(0, 1 << 32, a.size, dtype=np.uint64)
    words = np.empty(2 * a.size, np.uint32)
    words[0::2] = a.astype(np.uint32)
    words[1::2] = b.astype(np.uint32)
    want = oracle.box_muller(words)
    got64 = capi.lb_debug_box_muller(capi.LB_PREC_FP64, words)
    got32 = capi.lb_debug_box_muller(capi.LB_PREC_DEV32, words)
    assert np.max(np.abs(got64 - want)) < 1e-13
    err = np.abs(got32 - want)
    assert np.max(err) < 3e-6, (np.max(err), int(np.argmax(err)))
    assert capi.lb_debug_box_muller(capi.LB_PREC_DEV32, np.zeros(0, np.uint32)).size == 0
    # the kernels form two pairs at a time in packed instructions and an odd one alone: shifted
    # by one pair, every pair changes lane or form, and the values may not change
    shifted = capi.lb_debug_box_muller(capi.LB_PREC_DEV32, words[2:])
    np.testing.assert_array_equal(shifted, got32[2:])


@pytest.mark.parametrize("prec", ["fp64", "dev32"])
def test_correlations_of_a_batch(prec):
    """Sec. III.A-B real-space correlations <dphi(x, z) dphi(x, z')>_x and the Appendix A mixed
    correlations C(q_x, z, z') of every field, for each lattice of a heterogeneous batch, against
    the oracle.  FP32 deviations: within 1e-4 of the largest entry (the fields' own FP32
    representation, squared)."""
    ps = [LatticeParams(32, 16, kT=1e-4, G=0.5, grad_c0=0.3 / 16, seed=4, lattice_id=0),
          LatticeParams(64, 8, kT=2e-4, G=0.3, grad_c0=-0.2 / 8, seed=4, lattice_id=1)]
    fields = ("rho", "c", "ux", "uz")
    modes = [0, 1, 5]
    with Simulation(ps, precision=prec) as sim:
        sim.set_sampling(10, 4)
        sim.step(30)
        sim.set_correlations(fields, modes)  # counts from here: samples at 30, 34, ...
        sim.step(53)
        R = {(i, f): sim.correlation(f, lattice=i) for i in range(2) for f in fields}
        C = {(i, f, m): sim.mode_correlation(f, m, lattice=i) for i in range(2) for f in fields
             for m in range(len(modes))}
        with pytest.raises(capi.LBError):
            capi.lb_mode_correlation(sim.h, 0, 0, len(modes), np.empty((16, 16, 2)))
        sim.set_correlations(("c",))
        with pytest.raises(capi.LBError):  # not enabled any more
            sim.correlation("ux")
    for i, p in enumerate(ps):
        o = oracle_of(p)
        o.set_sampling(10, 4)
        o.step(30)
        o.set_correlations(fields, modes)
        o.step(53)
        for f in fields:
            want, n = o.correlation(f)
            got, ng = R[(i, f)]
            assert n == ng == 14
            tol = (1e-12 if prec == "fp64" else 1e-4) * np.abs(want).max()
            assert np.max(np.abs(got - want)) <= tol, (i, f, np.max(np.abs(got - want)), np.abs(want).max())
            for m in range(len(modes)):
                cw, _ = o.mode_correlation(f, m)
                cg, _ = C[(i, f, m)]
                # FP64: the bar of the structure factors (row transforms by FFT against direct sums)
                tol = (1e-9 if prec == "fp64" else 1e-4) * np.abs(cw).max()
                assert np.max(np.abs(cg - cw)) <= tol, (i, f, m)


@pytest.mark.parametrize("prec", ["fp64", "dev32"])
@pytest.mark.parametrize("shapes", [[(1, 2), (1, 5), (2, 2), (3, 3), (4, 2), (5, 7)],
                                    [(2, 2), (2, 5), (4, 2), (6, 3), (8, 7)]], ids=["generic", "bulk"])
def test_degenerate_lattices_in_one_batch(prec, shapes):
    """The smallest lattices the method allows, in one batch: one column (every link wraps onto
    the site itself), two and three columns, and two rows (both rows are wall rows, every vertical
    link is reflected).  Bulk copies need every width of the batch even, so the odd widths run the
    per-thread staging; the even batch runs the bulk copies, down to two columns, where both
    two-column halos are the lattice itself."""
    ps = [LatticeParams(Lx, Lz, lambda_s=1.1, lambda_d=0.9, kT=1e-4, G=0.4, grad_c0=0.3 / Lz, seed=8,
                        lattice_id=i) for i, (Lx, Lz) in enumerate(shapes)]
    with Simulation(ps, precision=prec) as sim:
        sim.step(60)
        got = [sim.populations(i) for i in range(len(ps))]
    for i, p in enumerate(ps):
        o = oracle_of(p)
        o.step(60)
        if prec == "fp64":
            assert_fp64_parity(got[i], o.populations())
        else:
            assert_dev32_parity(got[i], o.populations(), background(p.Lx, p.Lz, p.grad_c0))


@pytest.mark.parametrize("prec", ["fp64", "dev32"])
def test_bulk_strips_with_a_two_column_remainder(prec):
    """Bulk staging where the last strip holds two columns (Lx = tile + 2 and 2 tiles + 2): its
    right halo wraps to x = 0, 1 while the strips before it stage full windows (by tensor copies
    where they lie away from the x edges); per-step and persistent launches."""
    ps = [LatticeParams(130, 9, lambda_s=1.2, lambda_d=0.9, kT=1e-4, G=0.5, grad_c0=0.3 / 9, seed=31, lattice_id=0),
          LatticeParams(258, 6, lambda_s=1.2, lambda_d=0.9, kT=1e-4, G=0.5, grad_c0=0.2 / 6, seed=31, lattice_id=1)]
    oracles = []
    for p in ps:
        o = oracle_of(p)
        o.step(12)
        oracles.append(o.populations())
    for tile in [(128, 4), (64, 9)]:
        for kw in (dict(), dict(persistent=True)):
            with Simulation(ps, precision=prec, **kw) as sim:
                sim.set_tile(*tile)
                sim.step(12)
                got = [sim.populations(i) for i in range(len(ps))]
            for i, p in enumerate(ps):
                if prec == "fp64":
                    assert_fp64_parity(got[i], oracles[i])
                else:
                    assert_dev32_parity(got[i], oracles[i], background(p.Lx, p.Lz, p.grad_c0))


def test_device_memory_from_the_callers_allocator():
    """lb_create_batch_with_allocator with torch's caching allocator: the same results as the
    library's own allocations, torch accounts for the context's memory while it lives, and every
    buffer goes back when it is destroyed."""
    import torch

    p = LatticeParams(64, 32, kT=1e-4, G=0.5, grad_c0=0.3 / 32, seed=12)
    out = []
    for allocator in (None, "torch"):
        torch.cuda.synchronize()
        before = torch.cuda.memory_allocated()
        with Simulation(p, precision="dev32", allocator=allocator) as sim:
            sim.set_sampling(5, 5)
            sim.set_correlations(("c",), [1])
            sim.step(40)
            loss, grad = sim.pressure_shift_gradient(20, 10)
            held = torch.cuda.memory_allocated() - before
            nbytes = capi.lb_device_bytes(sim.h)
            out.append((sim.populations(), sim.structure_factor("c")[0], sim.correlation("c")[0], loss, grad))
        torch.cuda.synchronize()
        if allocator == "torch":
            assert held >= nbytes > 0
            assert torch.cuda.memory_allocated() == before
        else:
            assert held == 0
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)
