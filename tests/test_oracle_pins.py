"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks one oracle function against something other than itself: closed
forms (two-body orbits from the classical Kepler equation solved by bisection),
invariants (Newton's third law, conservation, time symmetry), finite differences,
convergence order, hand-computed values, and the paper's printed validation setup.
A plausible slip (a dropped term, a sign, a wrong coefficient, a transposed index)
fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import closed_forms as cf
import oracle as O
from paper_1208_1157_gb300 import ics

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
TWO_PI = 2 * math.pi


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def random_system(n, seed):
    rng = np.random.default_rng(seed)
    m = np.concatenate([[1.0], 10 ** rng.uniform(-5, -3, n - 1)])
    x = rng.normal(size=(n, 3)) * np.arange(1, n + 1)[:, None]
    v = rng.normal(size=(n, 3)) * 0.5
    return m, x, v


# ----------------------------------------------------------------- Eq. 1 + jerk
def test_accjerk_two_body_closed_form():
    m = np.array([1.0, 0.25])
    x = np.array([[0.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    v = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0]])
    a, j = O.accjerk(m, x, v)
    # a_1 = -m0 r/r^3 with r = (0, 2, 0): (0, -1/4, 0); a_0 = +m1 r/r^3 = (0, 1/16, 0)
    np.testing.assert_allclose(a, [[0, 0.0625, 0], [0, -0.25, 0]], rtol=0, atol=1e-16)
    # r.u = 0, so j_1 = -m0 u/r^3 = (-1/16, 0, 0), j_0 = m1 u / r^3 = (1/64, 0, 0)
    np.testing.assert_allclose(j, [[1 / 64, 0, 0], [-1 / 16, 0, 0]], rtol=0, atol=1e-16)


@pytest.mark.parametrize("n", [3, 5, 9])
def test_accjerk_newton_third_law(n):
    m, x, v = random_system(n, n)
    a, j = O.accjerk(m, x, v)
    scale_a = np.sum(np.abs(m[:, None] * a))
    scale_j = np.sum(np.abs(m[:, None] * j))
    assert np.max(np.abs(np.sum(m[:, None] * a, axis=0))) <= 1e-15 * scale_a
    assert np.max(np.abs(np.sum(m[:, None] * j, axis=0))) <= 1e-15 * scale_j


@pytest.mark.parametrize("n", [2, 4, 7])
def test_jerk_is_time_derivative_of_acceleration(n):
    m, x, v = random_system(n, 10 + n)
    _, j = O.accjerk(m, x, v)
    h = 1e-5
    ap = O.acc(m, x + h * v)
    am = O.acc(m, x - h * v)
    fd = (ap - am) / (2 * h)
    assert rel(fd, j) < 1e-8


def test_star_term_is_accumulated_last():
    # Sec. 4.2: the massive body's term is added after the planets' terms.  Six planet terms
    # of ~6e-17 each are lost if added to the star's 1.0 one by one, and survive if summed first.
    n = 8
    m = np.zeros(n)
    x = np.zeros((n, 3))
    m[0] = 1.0
    x[0] = [-1.0, 0, 0]          # star at distance 1 from the probe body 1
    x[1] = [0.0, 0, 0]
    m[1] = 1e-30
    for k in range(2, n):
        x[k] = [-float(k), 0, 0]
        m[k] = 6e-17 * k * k
    a, _ = O.accjerk(m, x, np.zeros((n, 3)))
    planets = 0.0
    for k in range(n - 1, 1, -1):
        planets += -m[k] / k ** 2
    assert a[1, 0] == planets + -1.0
    assert a[1, 0] != -1.0


def test_acc_matches_accjerk_and_brute_force():
    m, x, v = random_system(6, 3)
    a, _ = O.accjerk(m, x, v)
    brute = np.zeros_like(x)
    for i in range(6):
        for k in range(6):
            if k != i:
                r = x[k] - x[i]
                brute[i] += m[k] * r / np.linalg.norm(r) ** 3
    assert rel(a, brute) < 1e-14
    assert rel(O.acc(m, x), brute) < 1e-14


# ----------------------------------------------------------------- Hermite (Eqs. 3-4, Alg. 2)
def hermite_run(m, x, v, dt, steps, n_corr=2, form=O.CORR_KOKUBO):
    a, j = O.accjerk(m, x, v)
    for _ in range(steps):
        x, v, a, j = O.hermite_step(m, x, v, a, j, dt, n_corr, form)
    return x, v


def two_body_error(e, N, form=O.CORR_KOKUBO, periods=1.0):
    m0, m1 = 1.0, 1e-3
    mu = m0 + m1
    T = cf.period(mu, 1.0)
    sys_ = ics.two_body(1.0, e, m0, m1)
    x, v = hermite_run(sys_["mass"], sys_["pos"], sys_["vel"], periods * T / N, int(round(periods * N)), form=form)
    r_num = x[1] - x[0]
    r_ref, _ = cf.elliptic_at(mu, 1.0, e, 0.0, periods * T)
    return np.linalg.norm(r_num - r_ref)


@pytest.mark.parametrize("e", [0.0, 0.5])
def test_hermite_two_body_orbit_closes_after_one_period(e):
    # orbit closure to 1e-9 relative after one period with dt = T/4000
    assert two_body_error(e, 4000) <= 1e-9


@pytest.mark.parametrize("form", [O.CORR_KOKUBO, O.CORR_PRINTED])
def test_hermite_is_fourth_order(form):
    # e = 0.5 orbit, error at t = T against the closed form, dt halved twice
    errs = [two_body_error(0.5, N, form) for N in (500, 1000, 2000)]
    for a, b in zip(errs, errs[1:]):
        assert 13.0 <= a / b <= 19.0, errs


def test_printed_velocity_corrector_equals_time_symmetric_one():
    # Eq. 4's velocity update, based on the predicted state, is Kokubo's v-corrector
    m, x, v = random_system(4, 7)
    x = x * 3.0
    a, j = O.accjerk(m, x, v)
    dt = 0.01
    _, v1, _, _ = O.hermite_step(m, x, v, a, j, dt, 1, O.CORR_KOKUBO)
    _, v2, _, _ = O.hermite_step(m, x, v, a, j, dt, 1, O.CORR_PRINTED)
    assert rel(v2, v1) < 1e-14


def test_printed_form_coefficient_matters():
    # the printed 3/10 (instead of 3/20) would be a 2nd-order error term: the x update of
    # the two forms must differ by O(dt^5) only
    m = np.array([1.0, 0.5, 0.3])
    x = np.array([[0.0, 0, 0], [1.0, 0.2, 0], [-0.3, 1.1, 0.2]])
    v = np.array([[0.0, 0.1, 0], [0.1, 0.9, 0.1], [-0.8, 0.0, 0.0]])
    a, j = O.accjerk(m, x, v)
    d = []
    for dt in (0.04, 0.02):
        x1, _, _, _ = O.hermite_step(m, x, v, a, j, dt, 1, O.CORR_KOKUBO)
        x2, _, _, _ = O.hermite_step(m, x, v, a, j, dt, 1, O.CORR_PRINTED)
        d.append(np.max(np.abs(x1 - x2)))
    assert 24 <= d[0] / d[1] <= 40  # 2^5 = 32


def test_hermite_time_reversibility():
    # the time-symmetric corrector: N steps forward then N steps with -dt return to the start
    e = ics.three_body(4, seed=1)
    s = ics.subset(e, [0])
    m, x0, v0 = s["mass"], s["pos"], s["vel"]
    dt = TWO_PI * 1e-3
    errs = {}
    for nc in (1, 2, 8):
        x, v = hermite_run(m, x0, v0, dt, 100, nc)
        x, v = hermite_run(m, x, v, -dt, 100, nc)
        errs[nc] = max(rel(x, x0), rel(v, v0))
    assert errs[8] <= 1e-13
    assert errs[2] <= 1e-13
    assert errs[1] > errs[8]  # one correction is not converged: not exactly symmetric


def test_hermite_conservation_and_energy_order():
    e = ics.three_body(4, seed=1)
    s = ics.subset(e, [1])
    m, x0, v0 = s["mass"], s["pos"], s["vel"]
    E0, L0 = O.energy(m, x0, v0)
    # 1000 steps at the configured dt: E and L conserved to round-off level
    x, v = hermite_run(m, x0, v0, TWO_PI * 1e-3, 1000)
    E, L = O.energy(m, x, v)
    assert abs((E - E0) / E0) < 1e-12
    assert np.linalg.norm(L - L0) / np.linalg.norm(L0) < 1e-13
    # coarse steps expose the 4th-order energy error: halving dt divides it by ~16
    dE = []
    for dt in (TWO_PI / 50, TWO_PI / 100):
        x, v = hermite_run(m, x0, v0, dt, int(round(5 * TWO_PI / dt)))
        E, _ = O.energy(m, x, v)
        dE.append(abs((E - E0) / E0))
    assert dE[0] / dE[1] > 8.0, dE


# ----------------------------------------------------------------- Eq. 5 adaptive step
def test_adaptive_step_of_a_circular_two_body_orbit():
    # circular motion: a = -w^2 r, j = -w^2 v for both bodies, so |j|/|a| = w and
    # Eq. 5 gives tau / (sqrt(2) w) with w = sqrt(mu / a^3)
    m0, m1, a = 1.0, 1e-3, 1.7
    s = ics.two_body(a, 0.0, m0, m1)
    a0, j0 = O.accjerk(s["mass"], s["pos"], s["vel"])
    w = math.sqrt((m0 + m1) / a ** 3)
    assert O.adaptive_dt(a0, j0, 0.02) == pytest.approx(0.02 / (math.sqrt(2) * w), rel=1e-13)


def test_adaptive_hermite_lands_on_t_end_and_is_fourth_order_in_tau():
    m0, m1 = 1.0, 1e-3
    mu = m0 + m1
    T = cf.period(mu, 1.0)
    errs = []
    for tau in (0.02, 0.01, 0.005):
        s = ics.two_body(1.0, 0.5, m0, m1)
        out = O.integrate(s, T, tau, O.HERMITE_ADAPTIVE)
        assert out["time"][0] == T and out["status"][0] == O.DONE
        r_ref, _ = cf.elliptic_at(mu, 1.0, 0.5, 0.0, T)
        errs.append(np.linalg.norm(out["pos"][1] - out["pos"][0] - r_ref))
    for a, b in zip(errs, errs[1:]):
        assert 12.0 <= a / b <= 20.0, errs
    # backwards with a negative tau returns close to the start
    s = ics.two_body(1.0, 0.5, m0, m1)
    fwd = O.integrate(s, T / 3, 0.005, O.HERMITE_ADAPTIVE)
    back = O.integrate({**s, "pos": fwd["pos"], "vel": fwd["vel"]}, 0.0, -0.005, O.HERMITE_ADAPTIVE, time=fwd["time"])
    assert back["time"][0] == 0.0
    assert rel(back["pos"], s["pos"]) < 1e-9


# ----------------------------------------------------------------- Eq. 6, L
def test_energy_and_angular_momentum_hand_values():
    m = np.array([1.0, 0.5])
    x = np.array([[-1.0, 0, 0], [1.0, 0, 0]])
    v = np.array([[0, 1.0, 0], [0, -2.0, 0]])
    E, L = O.energy(m, x, v)
    # 1/2*1*1 + 1/2*0.5*4 - 1*0.5/2 (each pair once)
    assert E == pytest.approx(1.25, abs=1e-15)
    np.testing.assert_allclose(L, [0, 0, -2.0], atol=1e-15)
    m3 = np.array([2.0, 1.0, 1.0])
    x3 = np.array([[0, 0, 0], [3.0, 0, 0], [0, 4.0, 0]])
    v3 = np.zeros((3, 3))
    E3, _ = O.energy(m3, x3, v3)
    assert E3 == pytest.approx(-(2 / 3 + 2 / 4 + 1 / 5), abs=1e-15)


# ----------------------------------------------------------------- monitor
def test_monitor_cases():
    m = np.array([1.0, 1e-3, 1e-3])
    v = np.zeros((3, 3))
    x = np.array([[0, 0, 0], [1.0, 0, 0], [2.0, 0, 0]])
    assert O.monitor(m, x, v, 3.0, 100.0) == O.ACTIVE
    xe = x.copy()
    xe[2, 0] = 100.5
    assert O.monitor(m, xe, v, 3.0, 100.0) == O.EJECTED
    assert O.monitor(m, xe, v, 3.0, 0.0) == O.ACTIVE  # test switched off
    # planets at 1 and 1 + d on a line: R_H = k (2 + d)/2 with k = ((2e-3)/3)^(1/3); the
    # 3 R_H boundary is d = 3k / (1 - 1.5k)
    k = (2e-3 / 3) ** (1 / 3)
    d_crit = 3 * k / (1 - 1.5 * k)
    for fac, want in ((0.999, O.CLOSE_ENCOUNTER), (1.001, O.ACTIVE)):
        xc = np.array([[0, 0, 0], [1.0, 0, 0], [1.0 + fac * d_crit, 0, 0]])
        assert O.monitor(m, xc, v, 3.0, 100.0) == want
    xn = x.copy()
    xn[1, 1] = np.nan
    assert O.monitor(m, xn, v, 3.0, 100.0) == O.NONFINITE
    vn = v.copy()
    vn[2, 2] = np.inf
    assert O.monitor(m, x, vn, 0.0, 0.0) == O.NONFINITE


# ----------------------------------------------------------------- Stumpff / Kepler drift
@pytest.mark.parametrize("z", [-30.0, -5.0, -1.5, -1.0, -0.999, -0.3, 1e-9, 0.3, 0.999, 1.0, 1.5, 10.0, 30.0])
def test_stumpff_against_trig_closed_forms(z):
    c2, c3 = O.stumpff(z)
    if abs(z) < 1e-3:
        # closed forms cancel catastrophically here; the Taylor terms are exact to z^3
        e2, e3 = 0.5 - z / 24 + z * z / 720, 1 / 6 - z / 120 + z * z / 5040
        tol = 1e-15
    else:
        if z > 0:
            s = math.sqrt(z)
            e2, e3 = (1 - math.cos(s)) / z, (s - math.sin(s)) / (z * s)
        else:
            s = math.sqrt(-z)
            e2, e3 = (math.cosh(s) - 1) / (-z), (math.sinh(s) - s) / (-z * s)
        # the closed forms lose about log10(6/|z|) digits to cancellation
        tol = 6e-16 / min(abs(z), 1.0) + 2e-15
    assert c2 == pytest.approx(e2, rel=tol)
    assert c3 == pytest.approx(e3, rel=tol)


def test_stumpff_at_zero():
    assert O.stumpff(0.0) == (0.5, 1.0 / 6.0)


def _kepler_invariants(mu, r, v):
    return 0.5 * v @ v - mu / np.linalg.norm(r), np.cross(r, v)


@pytest.mark.parametrize("e,frac", [(0.0, 0.05), (0.3, 0.37), (0.9, 0.11), (0.6, 1.7)])
def test_kepler_drift_elliptic_matches_classical_kepler(e, frac):
    mu, a = 1.0, 1.3
    T = cf.period(mu, a)
    r0, v0 = cf.elliptic_state(mu, a, e, 0.4)
    r, v, st, it = O.kepler_drift(mu, r0, v0, frac * T)
    assert st == 0 and it < 20
    rr, vr = cf.elliptic_at(mu, a, e, 0.4, frac * T)
    assert rel(r, rr) < 1e-12 and rel(v, vr) < 1e-12


def test_kepler_drift_full_period_returns_to_start():
    mu, a, e = 1.2, 2.0, 0.2
    r0, v0 = cf.elliptic_state(mu, a, e, 1.1)
    r, v, st, _ = O.kepler_drift(mu, r0, v0, cf.period(mu, a))
    assert st == 0
    assert rel(r, r0) < 1e-12 and rel(v, v0) < 1e-12


@pytest.mark.parametrize("e,F0,t", [(1.5, -0.5, 3.0), (3.0, 0.2, 10.0), (1.01, 0.01, 2.0), (1.01, 0.01, -2.0)])
def test_kepler_drift_hyperbolic_matches_classical(e, F0, t):
    mu, a = 1.0, -2.0
    r0, v0 = cf.hyperbolic_state(mu, a, e, F0)
    r, v, st, _ = O.kepler_drift(mu, r0, v0, t)
    assert st == 0
    rr, vr = cf.hyperbolic_at(mu, a, e, F0, t)
    assert rel(r, rr) < 1e-11 and rel(v, vr) < 1e-11


@pytest.mark.parametrize("case", ["elliptic", "near_parabolic", "hyperbolic"])
def test_kepler_drift_invariants_and_composition(case):
    mu = 1.0
    r0 = np.array([1.0, 0.2, 0.1])
    speed = {"elliptic": 0.8, "near_parabolic": math.sqrt(2 / np.linalg.norm(r0)) * (1 + 1e-9), "hyperbolic": 2.0}[case]
    v0 = np.array([-0.1, 1.0, 0.05])
    v0 = v0 / np.linalg.norm(v0) * speed
    E0, h0 = _kepler_invariants(mu, r0, v0)
    r1, v1, s1, _ = O.kepler_drift(mu, r0, v0, 0.7)
    r2, v2, s2, _ = O.kepler_drift(mu, r1, v1, 1.9)
    r3, v3, s3, _ = O.kepler_drift(mu, r0, v0, 2.6)
    assert s1 == s2 == s3 == 0
    E3, h3 = _kepler_invariants(mu, r3, v3)
    # relative to the size of the two terms (E itself vanishes for the near-parabolic case)
    assert abs(E3 - E0) <= 1e-13 * (0.5 * v0 @ v0 + mu / np.linalg.norm(r0))
    assert rel(h3, h0) < 1e-13
    assert rel(r2, r3) < 1e-12 and rel(v2, v3) < 1e-12
    # and backwards: -dt undoes +dt
    rb, vb, sb, _ = O.kepler_drift(mu, r3, v3, -2.6)
    assert sb == 0 and rel(rb, r0) < 1e-12 and rel(vb, v0) < 1e-12


# ----------------------------------------------------------------- MVS coordinates
def test_dh_and_jacobi_round_trips():
    m, x, v = random_system(7, 21)
    for fwd, back in ((O.inertial_to_dh, O.dh_to_inertial), (O.inertial_to_jacobi, O.jacobi_to_inertial)):
        q, u = fwd(m, x, v)
        x2, v2 = back(m, q, u)
        assert rel(x2, x) < 1e-14 and rel(v2, v) < 1e-14


def test_jacobi_kinetic_energy_split():
    # T = 1/2 M V_cm^2 + sum_i 1/2 m'_i |w_i|^2 with reduced masses m'_i = m_i eta_{i-1}/eta_i
    m, x, v = random_system(6, 5)
    r, w = O.inertial_to_jacobi(m, x, v)
    eta = np.cumsum(m)
    T = 0.5 * eta[-1] * w[0] @ w[0] + sum(0.5 * m[i] * eta[i - 1] / eta[i] * w[i] @ w[i] for i in range(1, 6))
    assert T == pytest.approx(0.5 * np.sum(m * np.sum(v * v, axis=1)), rel=1e-14)
    # and the definition: r_i = x_i - centre of mass of bodies 0..i-1
    for i in range(1, 6):
        com = (m[:i, None] * x[:i]).sum(0) / m[:i].sum()
        assert rel(r[i], x[i] - com) < 1e-14


def test_dh_kinetic_energy_split():
    # democratic heliocentric: T = 1/2 M V^2 + sum_i>=1 P_i^2/(2 m_i) + |sum P_i|^2 / (2 m0)
    m, x, v = random_system(5, 6)
    q, u = O.inertial_to_dh(m, x, v)
    P = m[1:, None] * u[1:]
    T = 0.5 * m.sum() * u[0] @ u[0] + np.sum(np.sum(P * P, 1) / (2 * m[1:])) - P.sum(0) @ P.sum(0) / (2 * m[0]) * 0
    # the kinetic energy in DH variables carries the jump term with the opposite bookkeeping:
    # sum_i>=0 m_i |v_i - V|^2 / 2 = sum_i>=1 P_i^2/(2 m_i) + |sum_i>=1 P_i|^2/(2 m0)
    T = 0.5 * m.sum() * u[0] @ u[0] + np.sum(np.sum(P * P, 1) / (2 * m[1:])) + P.sum(0) @ P.sum(0) / (2 * m[0])
    assert T == pytest.approx(0.5 * np.sum(m * np.sum(v * v, axis=1)), rel=1e-13)
    assert rel(q[1:], x[1:] - x[0]) < 1e-14


def test_interaction_accelerations():
    # DH: planet-planet only; Jacobi: vanishes for two bodies (pure Kepler problem)
    m, x, v = random_system(4, 9)
    q, _ = O.inertial_to_dh(m, x, v)
    a = O.dh_interaction_acc(m, q)
    brute = np.zeros_like(q)
    for i in range(1, 4):
        for k in range(1, 4):
            if k != i:
                d = q[k] - q[i]
                brute[i] += m[k] * d / np.linalg.norm(d) ** 3
    assert rel(a, brute) < 1e-14
    m2, x2, v2 = random_system(2, 3)
    r2, _ = O.inertial_to_jacobi(m2, x2, v2)
    aj = O.jacobi_interaction_acc(m2, r2)
    assert np.max(np.abs(aj)) < 1e-15 * m2[0] / np.linalg.norm(r2[1]) ** 2


def test_jacobi_interaction_acceleration_is_minus_gradient():
    # the kick force is -dH_int/dr' divided by the reduced mass m'_i: finite differences of
    # H_int = -sum_{i<j} m_i m_j / r_ij + sum_i m0 m_i / |r'_i|
    m, x, v = random_system(4, 13)
    r, _ = O.inertial_to_jacobi(m, x, v)
    eta = np.cumsum(m)

    def h_int(rr):
        xx, _ = O.jacobi_to_inertial(m, rr, np.zeros_like(rr))
        U = 0.0
        for i in range(4):
            for k in range(i + 1, 4):
                U -= m[i] * m[k] / np.linalg.norm(xx[i] - xx[k])
        return U + sum(m[0] * m[i] / np.linalg.norm(rr[i]) for i in range(1, 4))

    a = O.jacobi_interaction_acc(m, r)
    for i in range(1, 4):
        mred = m[i] * eta[i - 1] / eta[i]
        for c in range(3):
            h = 1e-6
            rp, rm = r.copy(), r.copy()
            rp[i, c] += h
            rm[i, c] -= h
            g = (h_int(rp) - h_int(rm)) / (2 * h)
            assert -g / mred == pytest.approx(a[i, c], rel=1e-6, abs=1e-9)


# ----------------------------------------------------------------- MVS maps
def test_mvs_jacobi_two_body_is_exact_for_any_step():
    m0, m1 = 1.0, 1e-3
    s = ics.two_body(1.0, 0.3, m0, m1, E0=0.2)
    out = O.integrate(s, 7.3, 7.3 / 3, O.MVS_JACOBI)
    rr, vr = cf.elliptic_at(m0 + m1, 1.0, 0.3, 0.2, 7.3)
    x, v = out["pos"], out["vel"]
    assert rel(x[1] - x[0], rr) < 1e-12 and rel(v[1] - v[0], vr) < 1e-12


@pytest.mark.parametrize("kind", [O.MVS_DH, O.MVS_JACOBI])
@pytest.mark.parametrize("mscale", [1.0, 0.7])
def test_mvs_second_order_and_converges_to_hermite(kind, mscale):
    # cross-integrator validation of Sec. 5.2.1: MVS against a small-step Hermite solution
    # (mscale != 1 scales every mass, so a central mass of 1 cannot hide a missing 1/m0)
    s = ics.paper_standard(1, n=3)
    s["mass"] = s["mass"] * mscale
    t = 10 * math.pi / 5  # one inner orbit
    ref = O.integrate(s, t, t / 8000, O.HERMITE)
    errs = []
    for N in (200, 400, 800):
        out = O.integrate(s, t, t / N, kind)
        errs.append(rel(out["pos"], ref["pos"]))
    for a, b in zip(errs, errs[1:]):
        assert 3.5 <= a / b <= 4.5, errs
    assert errs[-1] < 1e-5


@pytest.mark.parametrize("kind", [O.MVS_DH, O.MVS_JACOBI])
def test_mvs_step_is_time_symmetric(kind):
    m, x, v = random_system(5, 31)
    x = x * 2 + np.sign(x)  # keep planets apart
    v = v * 0.2
    conv = O.inertial_to_dh if kind == O.MVS_DH else O.inertial_to_jacobi
    acc_f = O.dh_interaction_acc if kind == O.MVS_DH else O.jacobi_interaction_acc
    q, u = conv(m, x, v)
    a = acc_f(m, q)
    q1, u1, a1, st1 = O.mvs_step(kind, m, q, u, a, 0.05)
    q2, u2, _, st2 = O.mvs_step(kind, m, q1, u1, a1, -0.05)
    assert st1 == st2 == 0
    assert rel(q2, q) < 1e-13 and rel(u2, u) < 1e-13


def test_mvs_energy_error_bounded_without_secular_growth():
    # Table 1: the MVS energy error stays flat in time (5.0, 5.2, 5.1, 5.1 x 1e-11 at
    # 0.45..1.8 Mtu); here four equal windows of a shorter run at the paper's MVS dt
    flat = GOLDEN["table1_fractional_energy_error_x1e-11"]["mvs"]
    assert max(flat) / min(flat) < 1.1
    dt = GOLDEN["time_steps"]["mvs_dt"]
    s = ics.paper_standard(1, n=3)
    E0, _ = O.energy(s["mass"], s["pos"], s["vel"])
    out = O.integrate(s, 400.0, dt, O.MVS_DH, log_interval=10, log_cap=10000)
    err = np.abs(out["log"][0, : out["log_count"][0], 1] / E0 - 1)
    w = np.array_split(err, 4)
    peaks = [x.max() for x in w]
    assert max(peaks) / min(peaks) < 1.5, peaks


# ----------------------------------------------------------------- integration driver (Alg. 1)
def test_step_count_rule_and_last_step():
    s = ics.three_body(2, seed=3)
    dt = 0.01
    out = O.integrate(s, 0.0355, dt, O.HERMITE)  # 3 full steps + one of 0.0055
    assert np.all(out["time"] == 0.0355) and np.all(out["status"] == O.DONE)
    sub = ics.subset(s, [0])
    m, x, v = sub["mass"], sub["pos"], sub["vel"]
    a, j = O.accjerk(m, x, v)
    for h in (dt, dt, dt, 0.0355 - 3 * dt):
        x, v, a, j = O.hermite_step(m, x, v, a, j, h)
    assert rel(out["pos"][:3], x) < 1e-15
    # an integer number of steps within 1e-9 is taken exactly, no sliver step
    out2 = O.integrate(s, 1000 * dt, dt, O.HERMITE)
    x2, v2 = sub["pos"], sub["vel"]
    a, j = O.accjerk(m, x2, v2)
    for _ in range(1000):
        x2, v2, a, j = O.hermite_step(m, x2, v2, a, j, dt)
    assert rel(out2["pos"][:3], x2) == 0.0


def test_stop_then_untouched_and_logging():
    s = ics.three_body(3, seed=4)
    # put planet 2 of system 1 on an escape orbit from 90 AU
    s["pos"][5] = [90.0, 0, 0]
    s["vel"][5] = [1.0, 0, 0]
    out = O.integrate(s, 20.0, 0.01, O.HERMITE, eject_radius=100.0, log_interval=100, log_cap=50)
    assert list(out["status"]) == [O.DONE, O.EJECTED, O.DONE]
    t_stop = out["time"][1]
    assert 9.9 < t_stop < 10.1  # ~10 AU at unit speed
    assert out["log_count"][0] == 20 and out["log_count"][1] == int(t_stop / 1.0 + 1e-9)
    # the stopped system is not advanced again
    out2 = O.integrate({**s, "pos": out["pos"], "vel": out["vel"]}, 30.0, 0.01, O.HERMITE, eject_radius=100.0,
                       time=out["time"], status=out["status"])
    assert out2["time"][1] == t_stop
    assert rel(out2["pos"][3:6], out["pos"][3:6]) == 0.0
    assert out2["time"][0] == 30.0


# ----------------------------------------------------------------- Runge-Kutta Cash-Karp (Sec. 2.2.2)
def _rk_conditions(c, A, b):
    """Residuals of the 17 order conditions of an explicit Runge-Kutta method up to order 5
    (one per rooted tree, Butcher 2008, Sec. 31), grouped by order."""
    Ac = A @ c
    Ac2 = A @ c ** 2
    Ac3 = A @ c ** 3
    AAc = A @ Ac
    return {
        1: [b.sum() - 1],
        2: [b @ c - 1 / 2],
        3: [b @ c ** 2 - 1 / 3, b @ Ac - 1 / 6],
        4: [b @ c ** 3 - 1 / 4, b @ (c * Ac) - 1 / 8, b @ Ac2 - 1 / 12, b @ AAc - 1 / 24],
        5: [b @ c ** 4 - 1 / 5, b @ (c ** 2 * Ac) - 1 / 10, b @ (c * Ac2) - 1 / 15, b @ Ac ** 2 - 1 / 20,
            b @ (c * AAc) - 1 / 30, b @ Ac3 - 1 / 20, b @ (A @ (c * Ac)) - 1 / 40, b @ (A @ Ac2) - 1 / 60,
            b @ (A @ AAc) - 1 / 120],
    }


def test_rkck_tableau_satisfies_the_order_conditions():
    c, A, b5, b4 = O.rkck_tableau()
    assert np.all(np.triu(A) == 0.0)  # explicit
    assert np.abs(A.sum(axis=1) - c).max() < 1e-15  # row sums are the nodes
    r5 = _rk_conditions(c, A, b5)
    for order in range(1, 6):
        assert np.abs(r5[order]).max() < 2e-15, (order, r5[order])
    r4 = _rk_conditions(c, A, b4)
    for order in range(1, 5):
        assert np.abs(r4[order]).max() < 2e-15, (order, r4[order])
    # the embedded solution is only 4th order, so the difference estimates the local error
    assert np.abs(r4[5]).max() > 1e-4


def rkck_two_body_error(e, N, periods=1.0):
    m0, m1 = 1.0, 1e-3
    mu = m0 + m1
    T = cf.period(mu, 1.0)
    s = ics.two_body(1.0, e, m0, m1)
    out = O.integrate(s, periods * T, periods * T / N, O.RKCK)
    r_ref, _ = cf.elliptic_at(mu, 1.0, e, 0.0, periods * T)
    return np.linalg.norm(out["pos"][1] - out["pos"][0] - r_ref)


def test_rkck_fixed_step_is_fifth_order():
    # the propagated solution uses the 5th-order weights (local extrapolation)
    errs = [rkck_two_body_error(0.5, N) for N in (400, 800, 1600)]
    for a, b in zip(errs, errs[1:]):
        assert 26.0 <= a / b <= 38.0, errs


def test_rkck_error_vector_is_the_local_error_of_the_embedded_solution():
    m0, m1, e = 1.0, 1e-3, 0.5
    mu = m0 + m1
    T = cf.period(mu, 1.0)
    s = ics.two_body(1.0, e, m0, m1)
    ests = []
    for h in (T / 800, T / 1600):
        x5, v5, scaled, err = O.rkck_step(s["mass"], s["pos"], s["vel"], h)
        r_ref, u_ref = cf.elliptic_at(mu, 1.0, e, 0.0, h)
        r5, u5 = x5[1] - x5[0], v5[1] - v5[0]
        er, eu = err[1] - err[0], err[3] - err[2]
        # 4th-order solution = 5th-order one minus the error vector
        assert np.linalg.norm(r5 - er - r_ref) == pytest.approx(np.linalg.norm(er), rel=0.02)
        assert np.linalg.norm(u5 - eu - u_ref) == pytest.approx(np.linalg.norm(eu), rel=0.02)
        # the propagated 5th-order solution is one order better (error / estimate ~ h)
        assert np.linalg.norm(r5 - r_ref) < 0.2 * np.linalg.norm(er)
        # the scaled norm: largest body error over the largest body position / velocity
        X = np.linalg.norm(s["pos"], axis=1).max()
        V = np.linalg.norm(s["vel"], axis=1).max()
        want = max(np.linalg.norm(err[:2], axis=1).max() / X, np.linalg.norm(err[2:], axis=1).max() / V)
        assert scaled == pytest.approx(want, rel=1e-14)
        ests.append(scaled)
    assert 26.0 <= ests[0] / ests[1] <= 38.0  # local error O(h^5)


def test_rkck_adaptive_meets_the_tolerance_and_lands_on_t_end():
    m0, m1, e = 1.0, 1e-3, 0.5
    mu = m0 + m1
    T = cf.period(mu, 1.0)
    r_ref, _ = cf.elliptic_at(mu, 1.0, e, 0.0, T)
    res = {}
    for eps in (1e-9, 1e-11):
        s = ics.two_body(1.0, e, m0, m1)
        out = O.integrate(s, T, 0.01, O.RKCK_ADAPTIVE, rk_eps=eps, log_interval=1, log_cap=100000)
        assert out["time"][0] == T and out["status"][0] == O.DONE
        steps = int(out["log_count"][0])
        err = np.linalg.norm(out["pos"][1] - out["pos"][0] - r_ref)
        # each accepted step's local error is at most eps times the system's scale
        assert err <= 3.0 * steps * eps, (eps, err, steps)
        res[eps] = (steps, err)
    # steps grow like eps^(-1/5), the global error falls about in proportion to eps
    ratio = res[1e-11][0] / res[1e-9][0]
    assert 2.0 <= ratio <= 3.2, res
    assert res[1e-11][1] < res[1e-9][1] / 20, res


def test_rkck_adaptive_rejects_a_far_too_large_first_step():
    m0, m1 = 1.0, 1e-3
    s = ics.two_body(1.0, 0.3, m0, m1)
    T = cf.period(m0 + m1, 1.0)
    a = O.integrate(s, T / 2, 0.01, O.RKCK_ADAPTIVE, rk_eps=1e-12)
    b = O.integrate(s, T / 2, 50.0, O.RKCK_ADAPTIVE, rk_eps=1e-12)  # 16 periods: rejected until small
    assert a["status"][0] == b["status"][0] == O.DONE and b["time"][0] == T / 2
    assert rel(b["pos"], a["pos"]) < 1e-9
    # and backwards: the adaptive map integrates to an earlier time just as well
    back = O.integrate({**s, "pos": a["pos"], "vel": a["vel"]}, 0.0, -0.01, O.RKCK_ADAPTIVE, rk_eps=1e-12,
                       time=a["time"])
    assert back["time"][0] == 0.0 and rel(back["pos"], s["pos"]) < 1e-9


@pytest.mark.parametrize("L", [4.0, 0.25])
def test_rkck_step_obeys_kepler_scaling(L):
    # x -> L x, t -> L^(3/2) t, v -> L^(-1/2) v maps solutions of Eq. 1 (G = 1, masses fixed)
    # onto solutions: the step, its error vector and the scaled error norm must follow
    s = ics.three_body(1, seed=11)
    m, x, v = s["mass"], s["pos"], s["vel"]
    h = 0.05
    x5, v5, e5, err = O.rkck_step(m, x, v, h)
    xs, vs, es, errs = O.rkck_step(m, x * L, v / math.sqrt(L), h * L ** 1.5)
    assert rel(xs, x5 * L) < 1e-13 and rel(vs, v5 / math.sqrt(L)) < 1e-13
    assert rel(errs[:3], err[:3] * L) < 1e-9 and rel(errs[3:], err[3:] / math.sqrt(L)) < 1e-9
    assert es == pytest.approx(e5, rel=1e-9)


def test_rkck_adaptive_never_accepts_a_step_above_tolerance():
    # first trial = the whole interval, with a tolerance ten times below that step's error:
    # the trial must be rejected and the interval covered by smaller accepted steps
    m0, m1, e = 1.0, 1e-3, 0.5
    mu = m0 + m1
    T = cf.period(mu, 1.0)
    s = ics.two_body(1.0, e, m0, m1)
    h = T / 50
    _, _, big, _ = O.rkck_step(s["mass"], s["pos"], s["vel"], h)
    eps = big / 10
    out = O.integrate(s, h, h, O.RKCK_ADAPTIVE, rk_eps=eps, log_interval=1, log_cap=1000)
    steps = int(out["log_count"][0])
    assert out["time"][0] == h and steps >= 2
    r_ref, _ = cf.elliptic_at(mu, 1.0, e, 0.0, h)
    assert np.linalg.norm(out["pos"][1] - out["pos"][0] - r_ref) <= 3.0 * steps * eps


# ----------------------------------------------------------------- radial-velocity observable
def test_star_radial_velocity_of_a_circular_orbit():
    # circular two-body orbit seen at inclination i along z: the star moves on a circle of
    # speed m1/(m0+m1) sqrt(mu/a), half a turn out of phase with the planet, so its
    # z-velocity is -(m1/mu) sqrt(mu/a) sin(i) cos(n t + phase) for an orbit in the tilted
    # plane; the sign convention is rv = v_0 . los with los pointing away from the observer
    m0, m1, a, inc = 1.0, 1e-3, 1.3, 0.7
    mu = m0 + m1
    nmot = math.sqrt(mu / a ** 3)
    r = np.array([a, 0.0, 0.0])
    u = math.sqrt(mu / a) * np.array([0.0, math.cos(inc), math.sin(inc)])
    s = {"n_body": np.array([2], np.int32), "mass": np.array([m0, m1]),
         "pos": np.array([-m1 / mu * r, m0 / mu * r]), "vel": np.array([-m1 / mu * u, m0 / mu * u])}
    t_obs = np.linspace(0.1, 10.0, 9)
    out = O.observe_rv(s, t_obs, 1e-3, O.HERMITE, los=(0.0, 0.0, 1.0))
    want = -(m1 / mu) * math.sqrt(mu / a) * math.sin(inc) * np.cos(nmot * t_obs)
    assert np.abs(out["rv"][:, 0] - want).max() < 1e-12
    # the line of sight reverses the sign
    back = O.observe_rv(s, t_obs, 1e-3, O.HERMITE, los=(0.0, 0.0, -1.0))
    assert np.array_equal(back["rv"], -out["rv"])
