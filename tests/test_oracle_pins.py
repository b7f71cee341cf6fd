"""Pins of the oracle against what the paper and the mathematics fix (no GPU).

Each test names the passage it follows.  Together they are chosen so that a plausible
mistake in the oracle (a dropped term, a wrong sign or index, a transposed operand)
fails at least one of them.
"""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CZ = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _rest_state(Lx, Lz, rhoA, rhoB):
    f = np.empty((2, 9, Lz, Lx))
    for l in range(9):
        f[0, l] = W[l] * rhoA
        f[1, l] = W[l] * rhoB
    return f


# ---------------------------------------------------------------- noise generator
def test_philox_known_answers():
    """Philox4x32-10 of Salmon et al. (SC'11) against its published known-answer vectors."""
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def test_normals_are_standard():
    """Box-Muller normals of the noise stream: zero mean, unit variance, uncorrelated."""
    n = np.array([oracle.site_normals(7, 3, site, 11) for site in range(20000)])
    assert np.all(np.isfinite(n))
    assert abs(n.mean()) < 0.01
    assert abs(n.var() - 1.0) < 0.01
    c = np.corrcoef(n.T)
    assert np.max(np.abs(c - np.eye(16))) < 0.04
    # the counter words matter: another step, lattice or seed gives another stream
    assert not np.allclose(oracle.site_normals(7, 3, 5, 11), oracle.site_normals(7, 3, 5, 12))
    assert not np.allclose(oracle.site_normals(7, 3, 5, 11), oracle.site_normals(7, 4, 5, 11))
    assert not np.allclose(oracle.site_normals(7, 3, 5, 11), oracle.site_normals(8, 3, 5, 11))


def test_box_muller_word_roles_and_stream_wiring():
    """Box-Muller pairs (Sec. II.B noise): the first word of a pair sets the radius
    sqrt(-2 ln u1), the second the angle 2 pi u2, u = (2 (k mod 2^23) + 1) 2^-24 from the low 23
    bits; the site's sixteen normals are the pairs of its four Philox calls, counter (site, step,
    lattice, call) and key (seed low, seed high)."""
    # closed forms at the ends of the grid; the high bits are ignored
    n = oracle.box_muller([0xFF800000, 0x00000000, 0x007FFFFF, 0x003FFFFF])
    r0 = np.sqrt(48 * np.log(2.0))  # u1 = 2^-24
    r1 = np.sqrt(-2 * np.log1p(-2.0 ** -24))  # u1 = 1 - 2^-24
    ang0 = 2 * np.pi * 2.0 ** -24
    ang1 = 2 * np.pi * (0.5 - 2.0 ** -24)  # u2 = (2 (2^22 - 1) + 1) 2^-24
    np.testing.assert_allclose(n[:2], [r0 * np.cos(ang0), r0 * np.sin(ang0)], rtol=1e-14)
    np.testing.assert_allclose(n[2:], [r1 * np.cos(ang1), r1 * np.sin(ang1)], rtol=1e-9)
    assert n[3] > 0 and n[2] < 0
    # wiring of the site stream onto the Philox words
    seed, lid, site, step = (5 << 32) | 123, 9, 77, 4
    words = []
    for call in range(4):
        words += oracle.philox4x32_10([site, step, lid, call], [seed & 0xFFFFFFFF, seed >> 32])
    np.testing.assert_array_equal(oracle.site_normals(seed, lid, site, step), oracle.box_muller(words))


# ---------------------------------------------------------------- moment basis
def test_basis_is_weighted_orthogonal_with_golden_norms():
    """Table I basis: sum_l w_l T_al T_bl = N_a delta_ab (Eq. modes-discrete), N_a by hand."""
    T, w, N = oracle.basis()
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "d2q9_moment_norms.txt")) if not ln.startswith("#")]
    golden = np.array([int(r[1]) / int(r[2]) for r in rows])
    np.testing.assert_allclose(N, golden, rtol=4e-16, atol=0)
    np.testing.assert_allclose(w, W, rtol=0, atol=1e-16)
    gram = T @ np.diag(w) @ T.T
    np.testing.assert_allclose(gram, np.diag(golden), atol=1e-14)
    # brute force: the Table I polynomials evaluated on the links of Fig. 1
    c2 = CX ** 2 + CZ ** 2
    brute = np.array([np.ones(9), CX, CZ, 3 * c2 - 2, CX ** 2 - CZ ** 2, CX * CZ, (3 * c2 - 4) * CX,
                      (3 * c2 - 4) * CZ, 9 * c2 ** 2 - 15 * c2 + 2])
    np.testing.assert_array_equal(T, brute)
    # the inverse of Eq. (modes-discrete): f_l = w_l sum_a T_al m_a / N_a
    f = np.random.default_rng(0).random(9)
    m = T @ f
    np.testing.assert_allclose(w * (T.T @ (m / N)), f, atol=1e-15)


# ---------------------------------------------------------------- streaming and walls
def test_streaming_and_midway_bounce_back_by_hand():
    """With every lambda = 0 and no force or noise the collision is the identity, so one step
    is pure streaming (Eq. LB) with mid-way bounce-back at the walls (Sec. II.A).  A tagged
    population on link 5, c = (1, 1), is followed by hand on a 3 x 2 channel."""
    o = oracle.OracleLattice(3, 2, lambda_s=0, lambda_d=0, lambda_e=0, lambda_q=0, lambda_eps=0, kT=0, G=0,
                             grad_c0=0)
    base = _rest_state(3, 2, 0.5, 0.5)
    f = base.copy()
    f[0, 5, 0, 0] += 0.125  # species A, link 5, x = 0, z = 0
    f[1, 1, 1, 2] += 0.25   # species B, link 1, x = 2, z = 1 (crosses the periodic x edge)
    o.set_populations(f)
    expected = [  # (species, link, z, x) of each tag after steps 1..4
        [(0, 5, 1, 1), (1, 1, 1, 0)],
        [(0, 7, 1, 1), (1, 1, 1, 1)],  # link 5 reflected into link 7 at the top wall
        [(0, 7, 0, 0), (1, 1, 1, 2)],
        [(0, 5, 0, 0), (1, 1, 1, 0)],  # link 7 reflected into link 5 at the bottom wall
    ]
    for k in range(4):
        o.step(1)
        g = o.populations() - base
        e = np.zeros_like(g)
        e[expected[k][0]] = 0.125
        e[expected[k][1]] = 0.25
        np.testing.assert_allclose(g, e, atol=1e-15, err_msg=f"step {k + 1}")


def test_single_relaxation_gives_second_order_equilibrium():
    """With every lambda = 1 and no force or noise, Eq. (MRT) sends each species to the
    populations whose moments are m^eq of Table I, which are those of the second-order
    equilibrium w_l rho^S [1 + 3 c.U + 9/2 (c.U)^2 - 3/2 U^2] with the barycentric U
    (Eq. bar); the check is made on a random state, streamed by hand."""
    Lx, Lz = 4, 3
    rng = np.random.default_rng(1)
    f0 = _rest_state(Lx, Lz, 0.6, 0.4) * (1 + 0.2 * rng.standard_normal((2, 9, Lz, Lx)))
    o = oracle.OracleLattice(Lx, Lz, lambda_s=1, lambda_d=1, lambda_e=1, lambda_q=1, lambda_eps=1, kT=0, G=0,
                             grad_c0=0)
    o.set_populations(f0)
    o.step(1)
    got = o.populations()
    # stream by hand
    fs = np.empty_like(f0)
    opp = [0, 3, 4, 1, 2, 7, 8, 5, 6]
    for l in range(9):
        for z in range(Lz):
            for x in range(Lx):
                zs, xs = z - CZ[l], (x - CX[l]) % Lx
                fs[:, l, z, x] = f0[:, l, zs, xs] if 0 <= zs < Lz else f0[:, opp[l], z, x]
    rho = fs.sum(axis=1)
    jx = np.einsum("l,slzx->szx", CX, fs)
    jz = np.einsum("l,slzx->szx", CZ, fs)
    R = rho.sum(0)
    Ux, Uz = jx.sum(0) / R, jz.sum(0) / R
    for s in range(2):
        for l in range(9):
            cu = CX[l] * Ux + CZ[l] * Uz
            feq = W[l] * rho[s] * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (Ux ** 2 + Uz ** 2))
            np.testing.assert_allclose(got[s, l], feq, rtol=0, atol=1e-15)


# ---------------------------------------------------------------- conservation
def test_mass_conserved_per_species():
    """Per-species mass is conserved by every step (Sec. II, m^eq_0 = m_0; Sec. II.A)."""
    o = oracle.OracleLattice(16, 8, lambda_s=1.3, lambda_d=0.9, kT=1e-4, G=0.5, grad_c0=0.02, seed=3)
    m0 = o.mass()
    np.testing.assert_allclose(m0, [16 * 8 * 0.5, 16 * 8 * 0.5], rtol=5e-14)
    for _ in range(10):
        o.step(5)
        np.testing.assert_allclose(o.mass(), m0, rtol=5e-14, atol=0)


def test_noise_structure_and_variances():
    """Eqs. (noise-bin-expl) and (noise-bin-expl-high): xi_0 = 0, xi^A_{1,2} = -xi^B_{1,2}
    exactly; variances (2 - l_d) l_d kT rho^A rho^B / rho and 3 (2 - l_a) l_a N_a kT rho^S
    with the reference densities rho^S = 1/2 (hom); independent across species and moments."""
    lam = dict(lambda_s=1.1, lambda_d=0.7, lambda_e=1.3, lambda_q=0.9, lambda_eps=1.5)
    kT = 2.0
    o = oracle.OracleLattice(2, 2, kT=kT, G=0, grad_c0=0, seed=9, **lam)
    xi = np.array([o.site_noise(1, 0, t) for t in range(20000)])  # (n, 2, 9)
    assert np.all(xi[:, :, 0] == 0)
    assert np.all(xi[:, 0, 1:3] == -xi[:, 1, 1:3])
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "d2q9_moment_norms.txt")) if not ln.startswith("#")]
    N = np.array([int(r[1]) / int(r[2]) for r in rows])
    la = [None, lam["lambda_d"], lam["lambda_d"], lam["lambda_e"], lam["lambda_s"], lam["lambda_s"],
          lam["lambda_q"], lam["lambda_q"], lam["lambda_eps"]]
    ld = lam["lambda_d"]
    want_mom = (2 - ld) * ld * kT * 0.5 * 0.5 / 1.0
    for a in (1, 2):
        assert abs(xi[:, 0, a].var() / want_mom - 1) < 0.05
    for a in range(3, 9):
        want = 3 * (2 - la[a]) * la[a] * N[a] * kT * 0.5
        for s in range(2):
            assert abs(xi[:, s, a].var() / want - 1) < 0.05, (s, a)
    flat = xi[:, :, 1:].reshape(len(xi), 16)
    flat = np.delete(flat, [8, 9], axis=1)  # B momentum duplicates A momentum
    c = np.corrcoef(flat.T)
    assert np.max(np.abs(c - np.eye(14))) < 0.05


def test_noise_local_densities():
    """The loc variant (Sec. III.B) uses the local rho^S in the same variance formulas."""
    o = oracle.OracleLattice(2, 2, kT=1.0, lambda_s=1, lambda_d=1, lambda_e=1, lambda_q=1, lambda_eps=1,
                             noise_loc=True, seed=4)
    rA, rB = 0.8, 0.3
    o.set_populations(_rest_state(2, 2, rA, rB))
    xi = np.array([o.site_noise(0, 1, t) for t in range(20000)])
    assert abs(xi[:, 0, 1].var() / (rA * rB / (rA + rB)) - 1) < 0.05
    # a = 3: 3 (2 - 1) 1 N_3 kT rho^S with N_3 = 4
    assert abs(xi[:, 0, 3].var() / (12 * rA) - 1) < 0.05
    assert abs(xi[:, 1, 3].var() / (12 * rB) - 1) < 0.05


# ---------------------------------------------------------------- forces and pressure
def _resting(rhoA, rhoB):
    """Populations with all of rho^S on the rest link: streaming leaves them in place, so the
    pre-collision densities of the next step are rhoA, rhoB ([Lz, Lx]) and every j^S is zero,
    whence rho U = F / 2 (Eq. bar) with F the total force density."""
    Lz, Lx = rhoA.shape
    f = np.zeros((2, 9, Lz, Lx))
    f[0, 0], f[1, 0] = rhoA, rhoB
    return f


def test_fixed_wall_composition_ghosts_cancel_the_normal_force():
    """Sec. II.A wall ghosts of the non-ideal force (Eq. aNI), fixed-composition rule: beyond the
    bottom wall the ghost row holds the adjacent row's total density split c_0(-Lz/2) :
    1 - c_0(-Lz/2) between A and B, beyond the top wall c_0(+Lz/2) : 1 - c_0(+Lz/2).  The normal
    component of sum_l w_l c_l rho(r + c_l) at a wall row is (1/6) x (the row above minus the row
    below) for any x-dependence, so if the first interior row equals the ghost row the total
    normal force there vanishes and U_z = 0 (the gradient force cancels in the sum, Eq. NEcond;
    a* moves force between the species only).  The state below builds exactly that for both
    walls (c_0(-Lz/2) = 0.35, c_0(+Lz/2) = 0.65) with wall rows of other compositions: U_z must
    vanish at both wall rows under the fixed rule and not under the copy rule, and the rows
    that see no ghost must not depend on the rule."""
    Lx, Lz, g = 6, 4, 0.075
    cw_bot, cw_top = 0.5 - g * Lz / 2, 0.5 + g * Lz / 2
    rng = np.random.default_rng(5)
    rho0, rho3 = 0.9 + 0.2 * rng.random(Lx), 0.9 + 0.2 * rng.random(Lx)
    c_0, c_3 = 0.2 + 0.1 * rng.random(Lx), 0.75 + 0.1 * rng.random(Lx)  # far from the walls' values
    rhoA = np.stack([rho0 * c_0, rho0 * cw_bot, rho3 * cw_top, rho3 * c_3])
    rhoB = np.stack([rho0 * (1 - c_0), rho0 * (1 - cw_bot), rho3 * (1 - cw_top), rho3 * (1 - c_3)])
    fl = {}
    for fixed in (True, False):
        o = oracle.OracleLattice(Lx, Lz, G=0.7, kT=0, grad_c0=g, wall_fixed=fixed)
        o.set_populations(_resting(rhoA, rhoB))
        fl[fixed] = o.fields()
        np.testing.assert_allclose(fl[fixed]["rhoA"], rhoA, rtol=0, atol=1e-15)
    uz = fl[True]["uz"]
    assert np.max(np.abs(uz[[0, Lz - 1]])) < 1e-15, uz
    assert np.min(np.abs(fl[False]["uz"][[0, Lz - 1]])) > 1e-3, fl[False]["uz"]
    np.testing.assert_array_equal(fl[True]["uz"][1:Lz - 1], fl[False]["uz"][1:Lz - 1])
    np.testing.assert_array_equal(fl[True]["ux"][1:Lz - 1], fl[False]["ux"][1:Lz - 1])


def test_fixed_wall_composition_equals_copy_rule_at_the_wall_composition():
    """Sec. II.A: when the wall rows carry exactly the wall compositions c_0(-Lz/2) and
    c_0(+Lz/2), the fixed-composition ghosts equal the copied ones, so one step (noise on, so
    that every term of Eq. MRT enters) and the pre-collision pressure (Sec. III.C interaction
    part) agree between the two rules; on a state whose wall rows carry other compositions they
    differ.  (Those must not be 1/2: with a* the update depends on the ghosts only through the
    total force, whose ghost term rho^A(r) rho^B_ghost + rho^B(r) rho^A_ghost does not depend on
    how the ghost's density is split when c(r) = 1/2; so does the pressure's.)"""
    Lx, Lz, g = 8, 5, 0.05
    cw_bot, cw_top = 0.5 - g * Lz / 2, 0.5 + g * Lz / 2
    rng = np.random.default_rng(6)
    rho = 0.8 + 0.4 * rng.random((Lz, Lx))
    c = 0.3 + 0.4 * rng.random((Lz, Lx))
    c[0], c[Lz - 1] = cw_bot, cw_top
    res = {}
    for name, cc in (("at_cw", c), ("other", np.where(np.arange(Lz)[:, None] % (Lz - 1) == 0, 0.2, c))):
        for fixed in (True, False):
            o = oracle.OracleLattice(Lx, Lz, lambda_s=1.2, lambda_d=0.9, kT=1e-3, G=0.6, grad_c0=g, seed=4,
                                     wall_fixed=fixed)
            o.set_populations(_resting(rho * cc, rho * (1 - cc)))
            p = o.fields()["p"]
            o.step(1)
            res[name, fixed] = (o.populations(), p)
    for k in (0, 1):
        np.testing.assert_allclose(res["at_cw", True][k], res["at_cw", False][k], rtol=1e-14, atol=1e-16)
        assert np.max(np.abs(res["other", True][k] - res["other", False][k])) > 1e-4
    """Eq. (EQUATIONofSTATE): at rest and uniform, P = rho/3 + G rho^A rho^B / 3, and the
    uniform state is stationary (the non-ideal force vanishes)."""
    rA, rB, G = 0.6, 0.45, 0.7
    o = oracle.OracleLattice(6, 4, G=G, kT=0, grad_c0=0)
    f = _rest_state(6, 4, rA, rB)
    o.set_populations(f)
    p = o.fields()["p"]
    np.testing.assert_allclose(p, (rA + rB) / 3 + G * rA * rB / 3, rtol=0, atol=1e-15)
    o.step(3)
    np.testing.assert_allclose(o.populations(), f, rtol=0, atol=1e-15)


def test_gradient_forcing_cancels_in_total_momentum():
    """Eq. (NEcond): rho^A a^A_NE + rho^B a^B_NE = 0, so at G = 0 the rest state with the
    imposed profile c_0(z) has zero barycentric velocity although each species is pushed."""
    o = oracle.OracleLattice(5, 8, G=0, kT=0, grad_c0=0.03)
    fl = o.fields()
    assert np.max(np.abs(fl["ux"])) < 1e-16
    assert np.max(np.abs(fl["uz"])) < 1e-16
    # kinetic pressure of the rest state is rho/3 = 1/3 everywhere
    np.testing.assert_allclose(fl["p"], 1 / 3, atol=1e-15)


def _profile(o):
    fl = o.fields()
    c = fl["rhoA"] / (fl["rhoA"] + fl["rhoB"])
    Lz = c.shape[0]
    z = np.arange(Lz) + 0.5 - Lz / 2
    return c.mean(axis=1), 0.5 + z * o.params["grad_c0"]


def test_noiseless_ideal_mixture_keeps_linear_profile():
    """Sec. II: the gradient force fixes grad c = grad c_0 in the steady state; with G = 0 and
    no noise the linear profile c_0(z) = 1/2 + z grad_c0 holds at every row, walls included."""
    o = oracle.OracleLattice(4, 16, lambda_s=1.0, lambda_d=0.8, G=0, kT=0, grad_c0=0.01)
    o.step(4000)
    c, c0 = _profile(o)
    assert np.max(np.abs(c - c0)) < 1e-13
    fl = o.fields()
    assert np.max(np.abs(fl["uz"])) < 1e-15


def test_noiseless_nonideal_profile_with_astar():
    """Footnote to Eq. (ne-acc): with the a* correction the steady profile stays c_0(z) for
    G > 0 to the order of the lattice corrections; without it the profile is visibly off."""
    on = oracle.OracleLattice(4, 16, lambda_s=1.0, lambda_d=0.8, G=0.3, kT=0, grad_c0=0.01)
    off = oracle.OracleLattice(4, 16, lambda_s=1.0, lambda_d=0.8, G=0.3, kT=0, grad_c0=0.01, astar=False)
    on.step(3000)
    off.step(3000)
    c_on, c0 = _profile(on)
    c_off, _ = _profile(off)
    assert np.max(np.abs(c_on - c0)) < 1e-5
    assert np.max(np.abs(c_off - c0)) > 1e-3


def test_noiseless_pressure_is_flat_and_follows_eos():
    """Sec. III.C: the total pressure of the noiseless steady state is flat in z, and its
    mean is the equation of state (Eq. EQUATIONofSTATE) evaluated on the profile."""
    G = 0.3
    o = oracle.OracleLattice(4, 16, lambda_s=1.0, lambda_d=0.8, G=G, kT=0, grad_c0=0.01)
    o.step(3000)
    fl = o.fields()
    prof = fl["p"].mean(axis=1)
    assert np.ptp(prof[1:-1]) < 2e-5
    rho = fl["rhoA"] + fl["rhoB"]
    eos = rho / 3 + G * fl["rhoA"] * fl["rhoB"] / 3
    assert abs(fl["p"].mean() - eos.mean()) < 1e-5
    # G = 0: ideal gas, flat to round-off
    o0 = oracle.OracleLattice(4, 16, lambda_s=1.0, lambda_d=0.8, G=0, kT=0, grad_c0=0.01)
    o0.step(500)
    assert np.ptp(o0.fields()["p"]) < 1e-14


def test_profiles_are_time_averaged_row_means():
    """Sec. III.C profiles: with G = 0 and no noise the steady rows carry c_0(z), rho_bar, zero
    velocity and the ideal pressure rho_bar / 3 at every height; with noise and G > 0 the row
    means still sum to the conserved mass and their z-average is the mean pressure."""
    o = oracle.OracleLattice(4, 16, lambda_s=1.0, lambda_d=0.8, G=0, kT=0, grad_c0=0.01)
    o.step(4000)
    o.set_sampling(4000, 2)
    o.step(9)
    z = np.arange(16) + 0.5 - 8
    prof = {f: o.profile(f) for f in ("rho", "c", "ux", "uz", "p")}
    assert all(n == 5 for _, n in prof.values())
    np.testing.assert_allclose(prof["c"][0], 0.5 + 0.01 * z, rtol=0, atol=1e-13)
    # (the total mass carries ~1e-12 of accumulated round-off after 4000 steps)
    np.testing.assert_allclose(prof["rho"][0], 1.0, rtol=0, atol=1e-11)
    np.testing.assert_allclose(prof["p"][0], 1 / 3, rtol=0, atol=1e-11)
    assert np.ptp(prof["rho"][0]) < 1e-14 and np.ptp(prof["p"][0]) < 1e-14
    assert np.max(np.abs(prof["ux"][0])) < 1e-15 and np.max(np.abs(prof["uz"][0])) < 1e-15

    o = oracle.OracleLattice(8, 12, G=0.5, kT=1e-4, grad_c0=0.02, seed=3)
    o.set_sampling(10, 3)
    o.step(40)
    rho, n = o.profile("rho")
    assert n == 10
    assert abs(rho.sum() - 12.0) < 1e-13  # sum_z (1/Lx) sum_x rho = total mass / Lx
    p, _ = o.profile("p")
    _, p_avg, _ = o.mean_pressure()
    assert abs(p.mean() - p_avg) < 1e-14
    c, _ = o.profile("c")
    assert np.all(np.diff(c) > 0)  # the imposed gradient orders the rows


def test_correlations_obey_parseval_and_appendix_a():
    """Appendix A: the mode correlations C(q_x, z, z') = <dphi(q_x, z)^* dphi(q_x, z')> give the
    structure factor by the transform in z, S(q_x, q_z) = (1/Lz) sum_{z,z'} e^{i q_z (z - z')}
    C(q_x, z, z') (against the separately computed 2D power), and summed over every q_x they give
    the real-space correlation <dphi(x, z) dphi(x, z')>_x (Parseval); that one is symmetric with
    the field's mean square on its diagonal."""
    Lx, Lz = 8, 6
    o = oracle.OracleLattice(Lx, Lz, kT=1e-4, G=0.3, grad_c0=0.02, seed=3)
    o.set_sampling(2, 3)
    o.set_correlations(["rho", "c", "ux", "uz"], modes=range(Lx))
    o.step(12)
    z = np.arange(Lz)
    for f in ("rho", "c", "ux", "uz"):
        R, n = o.correlation(f)
        assert n == 4
        C = [o.mode_correlation(f, k)[0] for k in range(Lx)]
        np.testing.assert_allclose(sum(C).real / Lx, R, rtol=0, atol=1e-12 * np.abs(R).max())
        assert np.abs(sum(C).imag).max() < 1e-12 * np.abs(R).max()
        np.testing.assert_allclose(R, R.T, rtol=0, atol=1e-15 * np.abs(R).max())
        S, _ = o.structure_factor(f)
        for k in range(Lx):
            for nq in range(Lz):
                E = np.exp(1j * 2 * np.pi * nq / Lz * (z[:, None] - z[None, :]))
                v = (E * C[k]).sum() / Lz
                assert abs(v.imag) < 1e-12 * S.max() and abs(v.real - S[nq, k]) < 1e-12 * S.max(), (f, k, nq)
    # diagonal: the mean square per row, from the fields at the sample steps
    o2 = oracle.OracleLattice(Lx, Lz, kT=1e-4, G=0.3, grad_c0=0.02, seed=3)
    o2.step(5)
    fl = o2.fields()  # the pre-collision fields of step 5, which is sampled next
    o2.set_sampling(5, 1)
    o2.set_correlations(["c"])
    o2.step(1)
    zz = np.arange(Lz) + 0.5 - Lz / 2
    dc = fl["rhoA"] / (fl["rhoA"] + fl["rhoB"]) - (0.5 + 0.02 * zz)[:, None]
    R1, _ = o2.correlation("c")
    np.testing.assert_allclose(np.diag(R1), (dc ** 2).mean(axis=1), rtol=1e-12)


# ---------------------------------------------------------------- Fourier transform
def test_dft_power_single_mode_and_parseval():
    """Appendix: S(q) = |delta phi(q)|^2 with the unitary lattice transform.  A single plane
    wave puts L_x L_z / 4 at +q and -q; Parseval holds for any field."""
    Lx, Lz = 12, 6
    x = np.arange(Lx)[None, :]
    z = np.arange(Lz)[:, None]
    phi = np.cos(2 * np.pi * (3 * x / Lx + 2 * z / Lz))
    P = oracle.dft2_power(phi)
    e = np.zeros((Lz, Lx))
    e[2, 3] = e[Lz - 2, Lx - 3] = Lx * Lz / 4
    np.testing.assert_allclose(P, e, atol=1e-12)
    r = np.random.default_rng(2).standard_normal((Lz, Lx))
    assert abs(oracle.dft2_power(r).sum() - (r ** 2).sum()) < 1e-10
    # a field constant in x only has q_x = 0 power
    g = np.repeat(np.random.default_rng(3).standard_normal((Lz, 1)), Lx, axis=1)
    assert np.max(oracle.dft2_power(g)[:, 1:]) < 1e-20


# ---------------------------------------------------------------- statistical physics
def test_equilibrium_structure_factors_are_flat_fdt_values():
    """Sec. III.A, Eqs. (VELOCITY_EQ) and (CONCENTRATION_EQ): at grad c_0 = 0 the structure
    factors are flat, S_U = kT / rho_bar and S_c = 3 kT c_bar (1 - c_bar) / rho_bar = 0.75 kT
    (the density one, 3 kT rho_bar for an ideal gas of sound speed^2 1/3, is derived)."""
    kT = 1e-4
    o = oracle.OracleLattice(32, 16, lambda_s=1.0, lambda_d=1.0, lambda_e=1.0, lambda_q=1.0, lambda_eps=1.0,
                             kT=kT, G=0, grad_c0=0, seed=11)
    o.set_sampling(discard=500, every=4)
    o.step(500 + 4 * 2500)
    want = {"ux": kT, "uz": kT, "c": 0.75 * kT, "rho": 3 * kT}
    for fld, w in want.items():
        S, n = o.structure_factor(fld)
        assert n == 2500
        Sq = S.copy()
        Sq[0, 0] = np.nan  # q = 0 is fixed by conservation
        mean = np.nanmean(Sq)
        assert abs(mean / w - 1) < 0.02, (fld, mean / w)
        # flat: averaged along q_z (resp. q_x), every q_x (resp. q_z) bin within 10 %
        along_x = np.nanmean(Sq, axis=0)[1:]
        along_z = np.nanmean(Sq, axis=1)[1:]
        assert np.max(np.abs(along_x / w - 1)) < 0.1, (fld, along_x / w)
        assert np.max(np.abs(along_z / w - 1)) < 0.1, (fld, along_z / w)


@pytest.mark.slow
def test_nonequilibrium_concentration_spectrum_follows_the_prefactor_law():
    """Sec. III.B, Eqs. (decompose) and (prefactor): under an imposed gradient the concentration
    structure factor along the walls is S_c(q, 0) = 0.75 kT [1 + phi S_NE(qL)] with
    phi = (1/3) L^4 (grad c_0)^2 / (c_bar (1 - c_bar) (nu + D) D) and S_NE -> (qL)^-4 for qL >> 1,
    approached from below because of the confinement.  L = 16, Lx = 64, grad c_0 = 0.03,
    kT = 1e-4, every rate 1 (nu = D = 1/6, Eqs. diff and vis), eight seeds of 20000 steps (3000
    discarded, a sample every 20) on eight processes: the enhancement is large at the smallest
    qL (about 3.7, where the unbounded law would give 230), falls monotonically with q, its ratio
    to phi (qL)^-4 rises monotonically towards 1, and over qL = 7.9 .. 12.6 the enhancement
    summed is within a loose band (0.4 .. 1.2) of the law summed, with no fit; the velocity
    spectra keep the equilibrium value kT / rho_bar (Sec. III.B)."""
    Lx, Lz, g, kT = 64, 16, 0.03, 1e-4
    kw = dict(lambda_s=1.0, lambda_d=1.0, lambda_e=1.0, lambda_q=1.0, lambda_eps=1.0, kT=kT, G=0.0, grad_c0=g)
    jobs = [(dict(kw, seed=100 + i), Lx, Lz, 20000, 3000, 20, ("c", "ux", "uz")) for i in range(8)]
    res = oracle.sampled_runs(jobs, processes=8)
    assert all(r["c"][1] == 850 for r in res)
    Sc = np.array([r["c"][0][0] for r in res])  # q_z = 0, every q_x
    enh = Sc.mean(0) / (0.75 * kT) - 1
    nu = D = (1 / 1.0 - 0.5) / 3
    phi = (1 / 3) * Lz ** 4 * g ** 2 / (0.25 * (nu + D) * D)
    qt = 2 * np.pi * np.arange(Lx) / Lx * Lz
    law = np.zeros(Lx)
    law[1:] = phi * qt[1:] ** -4.0
    ratio = enh[1:7] / law[1:7]
    assert enh[1] > 2.0, enh[1]
    assert np.all(np.diff(enh[1:7]) < 0), enh[1:7]
    assert np.all(np.diff(ratio[:5]) > 0) and ratio[0] < 0.05, ratio
    k = np.arange(5, 9)
    band = enh[k].sum() / law[k].sum()
    assert 0.4 < band < 1.2, band
    for f in ("ux", "uz"):
        S = np.mean([r[f][0] for r in res], axis=0)
        S[0, 0] = np.nan
        assert abs(np.nanmean(S) / kT - 1) < 0.02, f


def test_openmp_build_gives_identical_results():
    """The same oracle source compiled with -fopenmp (its row loops on several host cores; used to
    time the oracle on every core) gives the plain build's results bit for bit: populations,
    structure factors, mean pressure and profiles, with noise, G > 0 and both wall rules."""
    threads = oracle.set_threads(4)
    assert threads == 4
    for fixed in (False, True):
        kw = dict(kT=1e-4, G=0.5, grad_c0=0.02, seed=3, wall_fixed=fixed, lambda_s=1.2, lambda_d=0.9)
        a, b = oracle.OracleLattice(32, 12, **kw), oracle.OracleLattice(32, 12, omp=True, **kw)
        for o in (a, b):
            o.set_sampling(3, 4)
            o.step(31)
        np.testing.assert_array_equal(a.populations(), b.populations())
        for f in ("rho", "c", "ux", "uz"):
            np.testing.assert_array_equal(a.structure_factor(f)[0], b.structure_factor(f)[0])
        assert a.mean_pressure() == b.mean_pressure()
        np.testing.assert_array_equal(a.profile("p")[0], b.profile("p")[0])
    oracle.set_threads(os.cpu_count() or 1)


# ---------------------------------------------------------------- gradient reference
def test_dual_number_gradient_matches_central_differences():
    """The gradient reference (forward-mode dual numbers through the oracle) against central
    differences of the oracle's own loss, on the same noise stream."""
    args = dict(kT=1e-3, G=0.5, grad_c0=0.05, seed=5, lambda_s=1.2, lambda_d=0.9, lambda_e=1.0)
    loss, g = oracle.pressure_shift_grad(8, 4, 30, **args)
    assert np.isfinite(loss) and abs(loss) > 0
    h = 1e-5
    fd = []
    for key in ("G", "lambda_s", "lambda_d"):
        up = dict(args, **{key: args[key] + h})
        dn = dict(args, **{key: args[key] - h})
        fd.append((oracle.pressure_shift(8, 4, 30, **up) - oracle.pressure_shift(8, 4, 30, **dn)) / (2 * h))
    fd = np.array(fd)
    np.testing.assert_allclose(g, fd, rtol=2e-4, atol=1e-10)
    assert abs(oracle.pressure_shift(8, 4, 30, **args) - loss) < 1e-15
