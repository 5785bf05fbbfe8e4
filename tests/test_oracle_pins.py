"""Pins of the CPU oracle against facts fixed by the paper and by the mathematics.

Nothing here compares the oracle with itself: every check is a closed form, a finite
difference of an independently pinned quantity, an invariant the paper states, a
brute-force evaluation in higher precision, or an independent integrator.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2210_02472_b300 import inputs
from tests import kepler


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# ----------------------------------------------------------------------------- acc
def test_acc_two_body_closed_form():
    rng = np.random.default_rng(1)
    for _ in range(5):
        pos = rng.normal(size=(3, 2))
        m = rng.uniform(0.1, 2.0, 2)
        a = oracle.acc(pos, m)
        d = pos[:, 1] - pos[:, 0]
        r = np.linalg.norm(d)
        assert rel(a[:, 0], m[1] * d / r ** 3) < 1e-15
        assert rel(a[:, 1], -m[0] * d / r ** 3) < 1e-15


def test_acc_momentum_balance():
    c = inputs.plummer(512, 11, imf="kroupa")
    a = oracle.acc(c.pos, c.mass)
    tot = np.abs((a * c.mass).sum(axis=1)).max()
    scale = np.abs(a * c.mass).sum()
    assert tot <= 1e-13 * scale


def test_acc_bruteforce_high_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    rng = np.random.default_rng(2)
    n = 9
    pos = rng.normal(size=(3, n))
    m = rng.uniform(0.1, 1.0, n)
    for eps2 in (0.0, 0.01):
        a = oracle.acc(pos, m, eps2=eps2)
        ref = np.zeros((3, n))
        for i in range(n):
            s = [mp.mpf(0)] * 3
            for j in range(n):
                if j == i:
                    continue
                d = [mp.mpf(pos[k, j]) - mp.mpf(pos[k, i]) for k in range(3)]
                r2 = d[0] ** 2 + d[1] ** 2 + d[2] ** 2 + mp.mpf(eps2)
                f = mp.mpf(m[j]) / (r2 * mp.sqrt(r2))
                s = [s[k] + f * d[k] for k in range(3)]
            ref[:, i] = [float(x) for x in s]
        err = np.abs(a - ref).max(axis=0) / np.linalg.norm(ref, axis=0)
        assert err.max() < 1e-14


def test_acc_additive_over_disjoint_sources():
    c = inputs.plummer(300, 12)
    A = np.arange(0, 100, dtype=np.int32)
    B1 = np.arange(100, 200, dtype=np.int32)
    B2 = np.arange(200, 300, dtype=np.int32)
    a12 = oracle.acc(c.pos, c.mass, A, np.concatenate([B1, B2]))
    a1 = oracle.acc(c.pos, c.mass, A, B1)
    a2 = oracle.acc(c.pos, c.mass, A, B2)
    assert rel(a12, a1 + a2) < 1e-13


def test_acc_coincident_is_error():
    pos = np.zeros((3, 3))
    pos[0, 2] = 1.0
    with pytest.raises(oracle.OracleError) as e:
        oracle.acc(pos, np.ones(3))
    assert e.value.code == oracle.ERR_COINCIDENT
    # softened: defined
    a = oracle.acc(pos, np.ones(3), eps2=1e-4)
    assert np.all(np.isfinite(a))


# ----------------------------------------------------------------------------- grad
def test_grad_two_body_closed_form():
    rng = np.random.default_rng(3)
    for _ in range(5):
        pos = rng.normal(size=(3, 2))
        m = rng.uniform(0.1, 2.0, 2)
        _, g = oracle.accel_grad(pos, m)
        d = pos[:, 1] - pos[:, 0]
        r = np.linalg.norm(d)
        M = m.sum()
        assert rel(g[:, 0], 2 * m[1] * M * d / r ** 6) < 1e-14
        assert rel(g[:, 1], -2 * m[0] * M * d / r ** 6) < 1e-14


@pytest.mark.parametrize("eps2", [0.0, 1e-3])
def test_grad_is_directional_derivative_of_acc(eps2):
    """G_i = d/dh a_i(x + h a) at h = 0 (the tidal tensor applied to a_j - a_i)."""
    c = inputs.plummer(64, 13, imf="kroupa")
    a, g = oracle.accel_grad(c.pos, c.mass, eps2=eps2)
    scale = np.linalg.norm(a, axis=0).max() / np.linalg.norm(g, axis=0).max()
    best = np.inf
    for hh in (1e-4, 3e-5, 1e-5):
        h = hh * scale
        ap = oracle.acc(c.pos + h * a, c.mass, eps2=eps2)
        am = oracle.acc(c.pos - h * a, c.mass, eps2=eps2)
        fd = (ap - am) / (2 * h)
        err = np.linalg.norm(fd - g, axis=0) / np.linalg.norm(g, axis=0)
        best = min(best, err.max())
    assert best < 1e-6


def test_grad_is_gradient_of_acceleration_norm():
    """G_i = (1 / (2 m_i)) grad_i sum_k m_k |a_k|^2  (the gradient potential)."""
    c = inputs.plummer(24, 14, imf="kroupa")
    _, g = oracle.accel_grad(c.pos, c.mass)

    def phi(pos):
        a = oracle.acc(pos, c.mass)
        return float((c.mass * (a * a).sum(axis=0)).sum())

    n = c.n
    fd = np.zeros((3, n))
    h = 1e-6
    for i in range(n):
        for k in range(3):
            p = c.pos.copy()
            p[k, i] += h
            fp = phi(p)
            p[k, i] -= 2 * h
            fm = phi(p)
            fd[k, i] = (fp - fm) / (2 * h) / (2 * c.mass[i])
    err = np.linalg.norm(fd - g, axis=0) / np.linalg.norm(g, axis=0)
    assert err.max() < 1e-5


def test_grad_momentum_balance():
    c = inputs.plummer(400, 15, imf="kroupa")
    _, g = oracle.accel_grad(c.pos, c.mass)
    tot = np.abs((g * c.mass).sum(axis=1)).max()
    assert tot <= 1e-12 * np.abs(g * c.mass).sum()


def test_cross_term_uses_inter_level_accelerations():
    """For disjoint S, F the gradient is the directional derivative of acc(S <- F) along
    the inter-level field (acc(S <- F) on S, acc(F <- S) on F), Sect. 2.2."""
    c = inputs.plummer(60, 16)
    S = np.arange(0, 40, dtype=np.int32)
    F = np.arange(40, 60, dtype=np.int32)
    aS, gS = oracle.accel_grad(c.pos, c.mass, S, F)
    aF, gF = oracle.accel_grad(c.pos, c.mass, F, S)
    field = np.zeros((3, c.n))
    field[:, S] = aS
    field[:, F] = aF
    h = 1e-5 * np.abs(aS).max() / np.abs(gS).max()
    fdS = (oracle.acc(c.pos + h * field, c.mass, S, F) - oracle.acc(c.pos - h * field, c.mass, S, F)) / (2 * h)
    fdF = (oracle.acc(c.pos + h * field, c.mass, F, S) - oracle.acc(c.pos - h * field, c.mass, F, S)) / (2 * h)
    assert (np.linalg.norm(fdS - gS, axis=0) / np.linalg.norm(gS, axis=0)).max() < 1e-6
    assert (np.linalg.norm(fdF - gF, axis=0) / np.linalg.norm(gF, axis=0)).max() < 1e-6
    # pairwise: the inter-level gradient kicks conserve momentum
    tot = (gS * c.mass[S]).sum(axis=1) + (gF * c.mass[F]).sum(axis=1)
    assert np.abs(tot).max() < 1e-12 * (np.abs(gS * c.mass[S]).sum() + np.abs(gF * c.mass[F]).sum())


def test_accel_grad_rejects_partial_overlap():
    c = inputs.plummer(20, 17)
    with pytest.raises(oracle.OracleError) as e:
        oracle.accel_grad(c.pos, c.mass, np.arange(0, 10), np.arange(5, 20))
    assert e.value.code == oracle.ERR_ARG


# ----------------------------------------------------------------------------- FSI
def kepler_error(e, nsteps, m2=0.5):
    m1 = 1.0
    pos, vel = kepler.binary(m1, m2, 1.0, e)
    T = kepler.period(m1, m2, 1.0)
    h = T / nsteps
    p, v = oracle.fsi_step(pos, vel, np.array([m1, m2]), h, steps=nsteps)
    x1, v1, x2, v2 = kepler.two_body_propagate(pos[:, 0], vel[:, 0], m1, pos[:, 1], vel[:, 1], m2, T)
    return max(np.abs(p[:, 0] - x1).max(), np.abs(p[:, 1] - x2).max())


def test_kepler_solver_pin():
    for e in (0.0, 0.3, 0.9, 0.999):
        for M in np.linspace(-7, 7, 29):
            E = kepler.kepler_E(M, e)
            assert abs(E - e * math.sin(E) - M) < 1e-13


def test_fsi_matches_kepler_closed_form_at_fourth_order():
    """Halving h cuts the error ~16x (fourth order, Sect. 2.1)."""
    errs = [kepler_error(0.5, n) for n in (200, 400, 800)]
    assert errs[-1] < 1e-6
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 13.0 < r1 < 19.0 and 13.0 < r2 < 19.0, (errs, r1, r2)


def test_fsi_time_reversible():
    c = inputs.plummer(64, 18)
    p1, v1 = oracle.fsi_step(c.pos, c.vel, c.mass, 1e-3, steps=20)
    p2, v2 = oracle.fsi_step(p1, -v1, c.mass, 1e-3, steps=20)
    assert np.abs(p2 - c.pos).max() < 1e-12
    assert np.abs(-v2 - c.vel).max() < 1e-11


def test_fsi_momentum_conserved():
    c = inputs.plummer(128, 19, imf="kroupa")
    p1, v1 = oracle.fsi_step(c.pos, c.vel, c.mass, 1e-3, steps=5)
    P0 = (c.vel * c.mass).sum(axis=1)
    P1 = (v1 * c.mass).sum(axis=1)
    assert np.abs(P1 - P0).max() < 1e-15 * np.abs(c.vel * c.mass).sum() + 1e-17


def test_fsi_three_body_against_dop853():
    """Burrau's three-body configuration (masses 3, 4, 5 at rest on a 3-4-5 triangle)
    integrated to t = 0.5 against scipy's DOP853 at rtol 1e-13."""
    from scipy.integrate import solve_ivp
    m = np.array([3.0, 4.0, 5.0])
    pos = np.array([[1.0, -2.0, 1.0], [3.0, -1.0, -1.0], [0.0, 0.0, 0.0]])
    vel = np.zeros((3, 3))

    def rhs(t, y):
        x = y[:9].reshape(3, 3)
        return np.concatenate([y[9:], oracle.acc(x, m).ravel()])

    sol = solve_ivp(rhs, (0, 0.5), np.concatenate([pos.ravel(), vel.ravel()]),
                    method="DOP853", rtol=1e-13, atol=1e-14)
    ref = sol.y[:9, -1].reshape(3, 3)
    p, v = oracle.fsi_step(pos, vel, m, 0.5 / 2000, steps=2000)
    assert np.abs(p - ref).max() < 1e-9


# ----------------------------------------------------------------------------- energy
def test_energy_two_body_and_plummer():
    pos = np.array([[0.0, 2.0], [0.0, 0.0], [0.0, 0.0]])
    vel = np.array([[0.0, 0.0], [1.0, -0.5], [0.0, 0.0]])
    m = np.array([1.0, 2.0])
    t, w = oracle.energy(pos, vel, m)
    assert t == pytest.approx(0.5 * 1 * 1 + 0.5 * 2 * 0.25, rel=1e-15)
    assert w == pytest.approx(-1.0 * 2.0 / 2.0, rel=1e-15)
    c = inputs.plummer(4096, 20)
    t, w = oracle.energy(c.pos, c.vel, c.mass)
    # Henon units: T = 1/4, W = -1/2 up to sampling noise and the 10 a truncation
    assert abs(t - 0.25) < 0.02 and abs(w + 0.5) < 0.03


def test_fsi_energy_error_fourth_order():
    c = inputs.plummer(32, 21)
    E0 = sum(oracle.energy(c.pos, c.vel, c.mass))
    dE = []
    for h in (2e-3, 1e-3):
        p, v = oracle.fsi_step(c.pos, c.vel, c.mass, h, steps=int(round(0.064 / h)))
        dE.append(abs(sum(oracle.energy(p, v, c.mass)) - E0))
    assert dE[0] / dE[1] > 8.0


# ----------------------------------------------------------------------------- steps
def test_timesteps_circular_binary_all_criteria_agree():
    """For a circular binary the free-fall and fly-by times coincide (Sect. 3.4), and
    |a|/|j| equals the same r/|v|."""
    m1, m2, a = 0.7, 0.3, 0.9
    pos, vel = kepler.binary(m1, m2, a, 0.0)
    tff = math.sqrt(a ** 3 / (m1 + m2))
    s_ff = oracle.timesteps(pos, vel, np.array([m1, m2]), eta_ff=1.0, eta_fb=1e9, eta_jerk=1e9)
    s_fb = oracle.timesteps(pos, vel, np.array([m1, m2]), eta_ff=1e9, eta_fb=1.0, eta_jerk=1e9)
    s_j = oracle.timesteps(pos, vel, np.array([m1, m2]), eta_ff=1e9, eta_fb=1e9, eta_jerk=1.0)
    for s in (s_ff, s_fb, s_j):
        assert np.allclose(s, tff, rtol=1e-13)


def test_gradient_and_velocity_acceleration_steps_circular_binary():
    """Sect. 3.4 criteria on a circular binary (COM frame, separation a, M = m1 + m2),
    from the two-body closed forms |a_1| = m2/a^2, |G_1| = 2 m2 M / a^5 (g' = G/24),
    |v_1| = (m2/M) (M/a)^{1/2} (and 1 <-> 2):
      velocity per acceleration  eta a^{3/2} M^{-1/2},
      gradient, first form       eta 12^{1/3} a^{3/2} M^{-1/2}  (the smaller of the two),
      gradient, second form      eta (12 a^3 / M)^{1/2}  (isolated by a large common
                                 velocity along z, which raises the other two)."""
    m1, m2, a = 0.7, 0.3, 0.9
    M = m1 + m2
    pos, vel = kepler.binary(m1, m2, a, 0.0)
    m = np.array([m1, m2])
    off = dict(eta_ff=1e30, eta_fb=1e30, eta_jerk=1e30)
    s_va = oracle.timesteps(pos, vel, m, eta_va=1.0, **off)
    assert np.allclose(s_va, a ** 1.5 / math.sqrt(M), rtol=1e-13)
    s_g = oracle.timesteps(pos, vel, m, eta_grad=1.0, **off)
    assert np.allclose(s_g, 12 ** (1 / 3) * a ** 1.5 / math.sqrt(M), rtol=1e-13)
    vz = vel.copy()
    vz[2] += 50.0
    s_g2 = oracle.timesteps(pos, vz, m, eta_grad=1.0, **off)
    assert np.allclose(s_g2, math.sqrt(12 * a ** 3 / M), rtol=1e-13)
    # the first gradient form with that velocity: eta (|v_i| 12 a^5 / (m_j M))^{1/3}
    vn = np.linalg.norm(vz, axis=0)
    first = (vn * 12 * a ** 5 / (m[::-1] * M)) ** (1 / 3)
    assert np.all(first > s_g2)
    s_min = oracle.timesteps(pos, vz, m, eta_grad=1.0, eta_va=1.0, **off)
    assert np.allclose(s_min, np.minimum(s_g2, vn * a ** 2 / m[::-1]), rtol=1e-13)


def test_gradient_steps_only_shrink_steps_and_deepen_the_hierarchy():
    """Adding criteria can only lower a particle's step (the step is a minimum), so an
    HHS interval with them keeps no more particles on the top level; the interval still
    conserves momentum (Sect. 2.2)."""
    c = inputs.plummer(200, 27, imf="kroupa")
    base = oracle.timesteps(c.pos, c.vel, c.mass)
    more = oracle.timesteps(c.pos, c.vel, c.mass, eta_grad=0.1, eta_va=0.1)
    assert np.all(more <= base) and np.any(more < base)
    tau = 1.0 / 32
    _, _, n0, _ = oracle.hhs_interval(c.pos, c.vel, c.mass, tau)
    p1, v1, n1, _ = oracle.hhs_interval(c.pos, c.vel, c.mass, tau, eta_grad=0.1, eta_va=0.1)
    assert n1[0] <= n0[0]
    P0 = (c.mass * c.vel).sum(axis=1)
    P1 = (c.mass * v1).sum(axis=1)
    assert np.abs(P1 - P0).max() <= 1e-14 * np.abs(c.mass * c.vel).sum()


def test_timesteps_jerk_is_time_derivative_of_acc():
    """The jerk criterion's j_i equals d/dt a_i(x + t v): with eta_ff = eta_fb = inf the
    step is eta |a| / |j| with j from a central difference of the oracle's acc."""
    c = inputs.plummer(40, 22, imf="kroupa")
    s = oracle.timesteps(c.pos, c.vel, c.mass, eta_ff=1e30, eta_fb=1e30, eta_jerk=1.0)
    a = oracle.acc(c.pos, c.mass)
    h = 1e-6
    j = (oracle.acc(c.pos + h * c.vel, c.mass) - oracle.acc(c.pos - h * c.vel, c.mass)) / (2 * h)
    ref = np.linalg.norm(a, axis=0) / np.linalg.norm(j, axis=0)
    assert rel(s, ref) < 1e-6


def test_timesteps_min_over_partners():
    """Free-fall step of a particle with one close neighbour is set by that pair."""
    pos = np.array([[0.0, 1e-3, 5.0, -4.0], [0.0, 0.0, 1.0, 2.0], [0.0, 0.0, 0.0, 1.0]])
    vel = np.zeros((3, 4))
    m = np.array([1.0, 2.0, 1.0, 1.0])
    s = oracle.timesteps(pos, vel, m, eta_ff=0.2, eta_fb=0.2, eta_jerk=1e30)
    assert s[0] == pytest.approx(0.2 * math.sqrt(1e-9 / 3.0), rel=1e-13)
    assert s[1] == pytest.approx(0.2 * math.sqrt(1e-9 / 3.0), rel=1e-13)


# ----------------------------------------------------------------------------- HHS
def test_hhs_all_slow_is_two_half_steps():
    """With every eps_i >= tau there is no fast set and the level is FSI(S, tau/2) twice."""
    c = inputs.plummer(48, 23)
    tau = 1e-3
    p, v, counts, _ = oracle.hhs_interval(c.pos, c.vel, c.mass, tau,
                                          fixed_steps=np.full(c.n, 1.0))
    p2, v2 = oracle.fsi_step(c.pos, c.vel, c.mass, tau / 2, steps=2)
    assert np.array_equal(p, p2) and np.array_equal(v, v2)
    assert counts[0] == c.n and counts[1:].sum() == 0


def test_hhs_depth_cap_zero_is_two_half_steps():
    """max_level = 0: the top level keeps every particle in S whatever its step (the depth
    cap), so the interval is FSI(all, tau/2) twice and reports the cap."""
    c = inputs.plummer(64, 25, imf="kroupa")
    tau = 1.0 / 8
    _, _, counts0, code0 = oracle.hhs_interval(c.pos, c.vel, c.mass, tau)
    assert counts0[1:].sum() > 0                      # uncapped, the set splits
    p, v, counts, code = oracle.hhs_interval(c.pos, c.vel, c.mass, tau, max_level=0,
                                             allow_maxlevel=True)
    p2, v2 = oracle.fsi_step(c.pos, c.vel, c.mass, tau / 2, steps=2)
    assert code == oracle.ERR_MAXLEVEL and code0 == oracle.OK
    assert np.array_equal(p, p2) and np.array_equal(v, v2)
    assert counts[0] == c.n


def test_hhs_momentum_conserved_and_levels():
    c = inputs.plummer(96, 24, imf="kroupa")
    tau = 1.0 / 16
    p, v, counts, _ = oracle.hhs_interval(c.pos, c.vel, c.mass, tau)
    assert counts[1:].sum() > 0          # a real hierarchy formed
    P0 = (c.vel * c.mass).sum(axis=1)
    P1 = (v * c.mass).sum(axis=1)
    assert np.abs(P1 - P0).max() < 1e-14 * np.abs(c.vel * c.mass).sum()
    E0 = sum(oracle.energy(c.pos, c.vel, c.mass))
    E1 = sum(oracle.energy(p, v, c.mass))
    assert abs((E1 - E0) / E0) < 1e-5


def _frozen_hierarchy_error(tau, nint):
    m = np.array([1.0, 0.3, 1e-2, 2e-2])
    pos, vel = kepler.binary(m[0], m[1], 0.1, 0.3)
    pos = np.concatenate([pos, np.array([[1.5, -2.0], [0.2, 0.5], [0.1, -0.3]])], axis=1)
    vel = np.concatenate([vel, np.array([[0.0, 0.1], [0.8, -0.6], [0.05, 0.0]])], axis=1)
    # binary two levels deeper than the outer bodies (steps tau/3 < tau/2)
    fixed = np.array([tau / 3, tau / 3, 2 * tau, 2 * tau])
    p, v = pos, vel
    for _ in range(nint):
        p, v, counts, _ = oracle.hhs_interval(p, v, m, tau, fixed_steps=fixed)
    assert counts[0] == 2 and counts[2] > 0
    return p


def test_hhs_frozen_hierarchy_fourth_order():
    """A frozen three-level hierarchy (inner binary two levels below two outer bodies)
    converges at fourth order only if the inter-level gradient kick uses the
    inter-level accelerations (Sect. 2.2)."""
    T = 0.4
    refp = _frozen_hierarchy_error(T / 256, 256)
    errs = []
    for k in (16, 32, 64):
        p = _frozen_hierarchy_error(T / k, k)
        errs.append(np.abs(p - refp).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 11.0 < r1 < 21.0 and 11.0 < r2 < 21.0, (errs, r1, r2)


# ----------------------------------------------------------------------------- PN1.0
def test_pn_test_particle_limit_is_schwarzschild_harmonic():
    """m_i -> 0, v_j = 0: the pair term reduces to the test-particle 1PN acceleration in
    harmonic coordinates, (M / (c^2 r^2)) [ (4 M / r - v^2) n + 4 (n.v) v ]."""
    rng = np.random.default_rng(5)
    c = 50.0
    for _ in range(5):
        x = rng.normal(size=3)
        v = rng.normal(size=3) * 0.3
        M = 1.3
        pos = np.stack([x, np.zeros(3)], axis=1)
        vel = np.stack([v, np.zeros(3)], axis=1)
        mass = np.array([1e-14, M])
        a = oracle.pn_acc(pos, vel, mass, np.array([0, 1]), c)
        r = np.linalg.norm(x)
        n = x / r
        ref = M / (c * c * r * r) * ((4 * M / r - v @ v) * n + 4 * (n @ v) * v)
        assert rel(a[:, 0], ref) < 1e-10


def test_pn_mask_only_pairs_with_a_black_hole():
    c = inputs.plummer(30, 25)
    bh = np.zeros(30, dtype=bool)
    a = oracle.pn_acc(c.pos, c.vel, c.mass, bh, 10.0)
    assert np.all(a == 0)
    bh[3] = True
    a = oracle.pn_acc(c.pos, c.vel, c.mass, bh, 10.0)
    assert np.all(a[:, 3] != 0) and np.count_nonzero(np.linalg.norm(a, axis=0)) == 30


def _lrl_angle(p, v, m):
    M = m.sum()
    r = p[:, 1] - p[:, 0]
    u = v[:, 1] - v[:, 0]
    L = np.cross(r, u)
    A = np.cross(u, L) / M - r / np.linalg.norm(r)
    return math.atan2(A[1], A[0])


@pytest.mark.parametrize("m2", [1.0, 1e-3])
def test_pn_periapsis_advance_rate(m2):
    """Two-body FSI + PN half-kicks: the periapsis advances by 6 pi G M / (c^2 a (1-e^2))
    per orbit (first term of Eq. secular_omega)."""
    m = np.array([1.0, m2])
    a0, e0, c = 1.0, 0.6, 200.0
    pos, vel = kepler.binary(m[0], m[1], a0, e0)
    T = kepler.period(m[0], m[1], a0)
    norb, nper = 6, 1000
    w0 = _lrl_angle(pos, vel, m)
    p, v = oracle.fsi_step(pos, vel, m, T / nper, c=c, is_bh=np.array([1, 1]),
                           steps=norb * nper)
    # finish at the same radial phase: step to the next apoapsis (max separation)
    def sep(pp):
        return np.linalg.norm(pp[:, 1] - pp[:, 0])
    best = (sep(p), p, v)
    for _ in range(60):
        p, v = oracle.fsi_step(p, v, m, T / nper, c=c, is_bh=np.array([1, 1]))
        if sep(p) > best[0]:
            best = (sep(p), p, v)
    w1 = _lrl_angle(best[1], best[2], m)
    dw = (math.remainder(w1 - w0, 2 * math.pi)) / norb
    expect = 6 * math.pi * m.sum() / (c * c * a0 * (1 - e0 * e0))
    assert dw == pytest.approx(expect, rel=0.02)


# ----------------------------------------------------------------------------- restarts
def _restart_reference(c, tau, k, **kw):
    """The interval re-run as attempt k of the restart procedure: every eta times 2^-k."""
    f = 0.5 ** k
    eta = {n: kw.get(n, d) * f for n, d in (("eta_ff", 0.2), ("eta_fb", 0.2), ("eta_jerk", 0.1),
                                           ("eta_grad", 0.0), ("eta_va", 0.0))}
    p, v, counts, _ = oracle.hhs_interval(c.pos, c.vel, c.mass, tau, allow_maxlevel=True, **eta)
    E0 = sum(oracle.energy(c.pos, c.vel, c.mass))
    return p, v, counts, abs((sum(oracle.energy(p, v, c.mass)) - E0) / E0)


def test_restart_within_tolerance_is_the_plain_interval():
    c = inputs.plummer(300, 28, imf="kroupa")
    p, v, counts, k, e, _ = oracle.hhs_interval_restart(c.pos, c.vel, c.mass, 1 / 16, 1.0)
    rp, rv, rc, re = _restart_reference(c, 1 / 16, 0)
    assert k == 0 and e == re
    assert np.array_equal(p, rp) and np.array_equal(v, rv) and np.array_equal(counts, rc)


def test_restart_halves_every_accuracy_parameter_per_restart():
    """Sect. 3.12: each consecutive restart lowers every time-step parameter by 50 %, until
    the energy error is within the tolerance; the accepted state is the interval run from
    the saved state with the parameters times 2^-k."""
    c = inputs.plummer(300, 28, imf="kroupa")
    kw = dict(eta_grad=0.1, eta_va=0.2)
    errs = [_restart_reference(c, 1 / 16, k, **kw)[3] for k in range(3)]
    assert errs[0] > errs[1] > errs[2]
    tol = (errs[1] * errs[2]) ** 0.5            # attempts 0 and 1 fail, attempt 2 passes
    p, v, counts, k, e, _ = oracle.hhs_interval_restart(c.pos, c.vel, c.mass, 1 / 16, tol, **kw)
    rp, rv, rc, re = _restart_reference(c, 1 / 16, 2, **kw)
    assert k == 2 and e == re
    assert np.array_equal(p, rp) and np.array_equal(v, rv) and np.array_equal(counts, rc)


def test_restart_keeps_the_current_result_when_the_error_grows():
    """A 24-body cluster whose error grows when the steps are halved (1.7e-5 -> 3.3e-5):
    with a 1e-6 tolerance the first restart's result is accepted."""
    c = inputs.plummer(24, 304, imf="kroupa")
    e0, e1 = (_restart_reference(c, 1 / 8, k)[3] for k in (0, 1))
    assert e1 > 1.5 * e0 > 1e-6
    p, v, counts, k, e, _ = oracle.hhs_interval_restart(c.pos, c.vel, c.mass, 1 / 8, 1e-6)
    rp, rv, _, re = _restart_reference(c, 1 / 8, 1)
    assert k == 1 and e == re
    assert np.array_equal(p, rp) and np.array_equal(v, rv)


def test_restart_stops_after_max_restarts():
    c = inputs.plummer(300, 28, imf="kroupa")
    p, v, counts, k, e, _ = oracle.hhs_interval_restart(c.pos, c.vel, c.mass, 1 / 16, 0.0,
                                                        max_restarts=3)
    rp, rv, _, re = _restart_reference(c, 1 / 16, 3)
    assert k == 3 and e == re
    assert np.array_equal(p, rp) and np.array_equal(v, rv)


# ----------------------------------------------------------------------------- subsystems
def _binary_and_perturbers():
    m1, m2, a, e = 0.02, 0.015, 0.05, 0.4
    bp, bv = kepler.binary(m1, m2, a, e)
    pp = np.array([[0.8, -0.3, 0.1], [-0.5, 0.9, -0.2], [0.1, -0.7, -0.9]]).T
    pv = np.random.default_rng(5).normal(0.0, 0.2, (3, 3))
    pos = np.concatenate([bp, pp], axis=1)
    vel = np.concatenate([bv, pv], axis=1)
    return pos, vel, np.array([m1, m2, 0.3, 0.25, 0.35])


def test_subsystem_step_of_an_isolated_binary_is_kepler_motion():
    """With the binary as the only subsystem and no other particle, every kick vanishes and
    Algorithm 1 reduces to its two subsystem flows of eps/2: the exact two-body motion."""
    m1, m2 = 0.6, 0.4
    pos, vel = kepler.binary(m1, m2, 0.05, 0.7)
    p, v = oracle.fsi_step_sub(pos, vel, np.array([m1, m2]), [[0, 1]], 3e-3, steps=10)
    x1, v1, x2, v2 = kepler.two_body_propagate(pos[:, 0], vel[:, 0], m1, pos[:, 1], vel[:, 1],
                                               m2, 0.03)
    assert np.abs(p[:, 0] - x1).max() <= 1e-13 * np.abs(x1).max()
    assert np.abs(p[:, 1] - x2).max() <= 1e-13 * np.abs(x2).max()
    assert np.abs(v[:, 0] - v1).max() <= 1e-13 * np.abs(v1).max()
    assert np.abs(v[:, 1] - v2).max() <= 1e-13 * np.abs(v2).max()


def test_masked_sums_leave_out_only_the_partner():
    """acc' and G' of a subsystem member equal the plain sums over every source except its
    partner; singles keep the plain sums."""
    c = inputs.plummer(40, 29, imf="kroupa")
    pairs = [[3, 17], [8, 30]]
    partner = {3: 17, 17: 3, 8: 30, 30: 8}
    field = inputs.random_field(40, 30)
    a = oracle.acc_sub(c.pos, c.mass, pairs)
    g = oracle.grad_sub(c.pos, c.mass, pairs, field)
    for i in range(40):
        B = [j for j in range(40) if j != partner.get(i, -1)]
        ai = oracle.acc(c.pos, c.mass, [i], B)
        gi = oracle.grad(c.pos, c.mass, field, [i], B)
        assert np.allclose(a[:, [i]], ai, rtol=1e-14, atol=0)
        assert np.allclose(g[:, [i]], gi, rtol=1e-13, atol=0)


def test_subsystem_step_is_fourth_order_and_conserves_momentum():
    """A binary subsystem (a = 0.05, e = 0.4) with three perturbers against a DOP853
    solution of the full five-body problem (rtol 1e-13): halving eps cuts the position
    error ~16x (Algorithm 1 keeps the FSI's order: the intra-subsystem potential commutes
    with U', so the gradient term is unchanged); total momentum is conserved."""
    from scipy.integrate import solve_ivp
    pos, vel, m = _binary_and_perturbers()
    N, T = 5, 0.25

    def rhs(t, y):
        x = y[:15].reshape(3, N)
        acc = np.zeros((3, N))
        for i in range(N):
            for j in range(N):
                if i != j:
                    d = x[:, j] - x[:, i]
                    acc[:, i] += m[j] * d / np.linalg.norm(d) ** 3
        return np.concatenate([y[15:], acc.ravel()])

    sol = solve_ivp(rhs, (0, T), np.concatenate([pos.ravel(), vel.ravel()]), method="DOP853",
                    rtol=1e-13, atol=1e-16)
    ref = sol.y[:15, -1].reshape(3, N)
    errs = []
    for k in (16, 32, 64):
        p, v = oracle.fsi_step_sub(pos, vel, m, [[0, 1]], T / k, steps=k)
        errs.append(np.abs(p - ref).max())
        assert np.abs((m * v).sum(axis=1) - (m * vel).sum(axis=1)).max() <= 1e-15
    for r in (errs[0] / errs[1], errs[1] / errs[2]):
        assert 12.0 < r < 20.0, errs


# ----------------------------------------------------------------------------- kick / drift
def test_kick_drift_exact_dyadic_closed_form():
    """v' = v + c_k a and x' = x + c_d v' on dyadic numbers, where every operation is
    exact: the oracle must reproduce the closed form bit for bit, only on the listed ids."""
    pos = np.array([[1.5, -2.0, 0.75], [0.25, 4.0, -1.0], [3.0, 0.5, 2.0]])
    vel = np.array([[0.25, 1.0, -0.5], [-0.75, 0.0, 2.0], [0.5, -1.5, 0.125]])
    P = np.array([2, 0], dtype=np.int32)
    acc = np.array([[-2.0, 4.0], [1.0, 0.5], [0.0, -8.0]])     # rows for ids 2, 0
    ck, cd = 0.5, 0.125
    p, v = oracle.kick_drift(pos, vel, acc, ck, cd, P)
    ev, ex = vel.copy(), pos.copy()
    for k, i in enumerate(P):
        ev[:, i] = vel[:, i] + ck * acc[:, k]
        ex[:, i] = pos[:, i] + cd * ev[:, i]
    assert np.array_equal(v, ev) and np.array_equal(p, ex)
    assert v[0, 2] == -0.5 - 1.0 and p[0, 2] == 0.75 + 0.125 * -1.5
    assert np.array_equal(p[:, 1], pos[:, 1]) and np.array_equal(v[:, 1], vel[:, 1])
    # drift only: x + c_d v
    p2, v2 = oracle.kick_drift(pos, vel, None, 0.0, 0.25)
    assert np.array_equal(v2, vel) and np.array_equal(p2, pos + 0.25 * vel)


def test_fsi_cycle_is_its_kick_and_drift_factors():
    """Eq. fsi-cycle as a product of kicks and drifts: kick h/6 (a), drift h/2, kick 2h/3
    with a + (h^2/24) G, drift h/2, kick h/6 (a), each a from the current positions,
    composed from the oracle's kick_drift, acc and grad, equals the oracle's fsi_step."""
    c = inputs.plummer(40, 31, imf="kroupa")
    h = 1e-3
    x, v = c.pos.copy(), c.vel.copy()
    a = np.asarray(oracle.acc(x, c.mass))
    x, v = oracle.kick_drift(x, v, a, h / 6, h / 2)
    a = np.asarray(oracle.acc(x, c.mass))
    G = np.asarray(oracle.grad(x, c.mass, a))
    x, v = oracle.kick_drift(x, v, a + h * h / 24 * G, 2 * h / 3, h / 2)
    a = np.asarray(oracle.acc(x, c.mass))
    x, v = oracle.kick_drift(x, v, a, h / 6, 0.0)
    rp, rv = oracle.fsi_step(c.pos, c.vel, c.mass, h)
    assert np.abs(x - rp).max() <= 1e-15 * np.abs(rp).max()
    assert np.abs(v - rv).max() <= 1e-14 * np.abs(rv).max()
