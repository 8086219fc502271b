"""GPU parity of the MVS path (democratic heliocentric and Jacobi) against the oracle."""
import math

import numpy as np
import pytest

import closed_forms as cf
import oracle as O
from gpu_util import TWO_PI, assert_parity, oracle_sensitivity, run_gpu, run_oracle
from paper_1208_1157_gb300 import ics

pytestmark = pytest.mark.gpu

DT = TWO_PI / 20  # 1/20 of the inner period


@pytest.mark.parametrize("kind", [O.MVS_DH, O.MVS_JACOBI])
def test_compact_eight_body_parity_1000_steps(kind):
    ens = ics.mvs_compact(256, seed=4)
    o = run_oracle(ens, 1000 * DT, kind, DT, ce=3.0, ej=100.0)
    sens = oracle_sensitivity(ens, 1000 * DT, kind, DT, ce=3.0, ej=100.0)
    g = run_gpu(ens, 1000 * DT, kind, DT, ce=3.0, ej=100.0)
    assert_parity(ens, g, o, sens=sens)
    # warm-started Newton: between one and (on average) a handful of iterations per solve
    solves = 7 * int(np.sum(np.round(o["time"] / DT)))
    assert solves <= g["stats"]["kepler_iterations"] <= 6 * solves


@pytest.mark.parametrize("kind", [O.MVS_DH, O.MVS_JACOBI])
def test_wide_spaced_eight_body_parity_1000_steps(kind):
    # planets 6 to 8 mutual Hill radii apart: most systems run the whole 1000 steps (234 of
    # 256), and at least 90 % of those meet the strict 1e-10 bar (assert_parity's cap)
    ens = ics.mvs_compact(256, seed=16, k_lo=6.0, k_hi=8.0)
    o = run_oracle(ens, 1000 * DT, kind, DT, ce=3.0, ej=100.0)
    sens = oracle_sensitivity(ens, 1000 * DT, kind, DT, ce=3.0, ej=100.0)
    g = run_gpu(ens, 1000 * DT, kind, DT, ce=3.0, ej=100.0)
    assert int(np.sum(o["status"] <= 1)) >= 200
    assert_parity(ens, g, o, sens=sens)


@pytest.mark.parametrize("kind", [O.MVS_DH, O.MVS_JACOBI])
def test_ragged_mvs_parity(kind):
    ens = ics.ragged(300, seed=12)
    o = run_oracle(ens, 300 * DT, kind, DT, ce=3.0, ej=100.0)
    sens = oracle_sensitivity(ens, 300 * DT, kind, DT, ce=3.0, ej=100.0)
    g = run_gpu(ens, 300 * DT, kind, DT, ce=3.0, ej=100.0)
    assert_parity(ens, g, o, sens=sens, steps=300)


def test_jacobi_two_body_exact():
    m0, m1 = 1.0, 1e-3
    s = ics.two_body(1.0, 0.3, m0, m1, E0=0.2)
    ens = ics.concat(*[s] * 40)
    g = run_gpu(ens, 7.3, O.MVS_JACOBI, 7.3 / 3)
    rr, vr = cf.elliptic_at(m0 + m1, 1.0, 0.3, 0.2, 7.3)
    for k in range(40):
        x, v = g["pos"][2 * k:2 * k + 2], g["vel"][2 * k:2 * k + 2]
        assert np.max(np.abs(x[1] - x[0] - rr)) <= 1e-12 * np.max(np.abs(rr))
        assert np.max(np.abs(v[1] - v[0] - vr)) <= 1e-12 * np.max(np.abs(vr))


@pytest.mark.parametrize("kind", [O.MVS_DH, O.MVS_JACOBI])
def test_mvs_shortened_last_step_and_log(kind):
    ens = ics.mvs_compact(64, seed=13)
    t1 = 77.3 * DT
    o = run_oracle(ens, t1, kind, DT, log_interval=10, log_cap=10)
    g = run_gpu(ens, t1, kind, DT, log_interval=10, log_cap=10)
    assert_parity(ens, g, o)
    for s in range(64):
        lo = o["log"][s, : o["log_count"][s]]
        np.testing.assert_allclose(g["logs"][s][:, 1], lo[:, 1], rtol=1e-11)


def test_mvs_full_size_sampled():
    # 16384 x 8 bodies in the benchmark's launch configuration; 2000 steps, 24 samples
    ens = ics.mvs_compact(16384, seed=4)
    g = run_gpu(ens, 2000 * DT, O.MVS_JACOBI, DT, ce=3.0, ej=100.0)
    idx = np.sort(np.random.default_rng(2).choice(16384, 24, replace=False))
    sub = ics.subset(ens, idx)
    o = run_oracle(sub, 2000 * DT, O.MVS_JACOBI, DT, ce=3.0, ej=100.0)
    sens = oracle_sensitivity(sub, 2000 * DT, O.MVS_JACOBI, DT, ce=3.0, ej=100.0)
    gs = {"pos": g["pos"].reshape(-1, 8, 3)[idx].reshape(-1, 3), "vel": g["vel"].reshape(-1, 8, 3)[idx].reshape(-1, 3),
          "time": g["time"][idx], "status": g["status"][idx]}
    assert_parity(sub, gs, o, sens=sens)


@pytest.mark.parametrize("kind", [O.MVS_DH, O.MVS_JACOBI])
def test_mvs_chunked_launches(kind):
    from paper_1208_1157_gb300 import swarm as S

    ens = ics.mvs_compact(64, seed=14)
    ref = run_gpu(ens, 300 * DT, kind, DT, ce=3.0, ej=100.0)
    with S.Ensemble(ens) as e:
        e.set_stop(3.0, 100.0)
        e.set_option(S.OPT_STEPS_PER_LAUNCH, 50)
        e.integrate(300 * DT, kind, DT)
        # six chunks, each after the launch that compacts the bin to its runnable systems
        assert e.stats()["kernel_launches"] == 12
        got = e.state()
    from gpu_util import per_system_errors
    assert np.array_equal(got["status"], ref["status"])
    ex, ev = per_system_errors(ens, got, ref)
    assert ex.max() <= 1e-10 and ev.max() <= 1e-10


@pytest.mark.parametrize("kind", [O.MVS_DH, O.MVS_JACOBI])
def test_mvs_backward_parity_and_return(kind):
    # negative steps (t_end < t): parity with the oracle, and the symmetric map brought
    # back to its start by the same number of steps of -dt
    from paper_1208_1157_gb300 import swarm as S
    from gpu_util import per_system_errors

    ens = ics.mvs_compact(128, seed=15)
    o = run_oracle(ens, -200 * DT, kind, -DT)
    sens = oracle_sensitivity(ens, -200 * DT, kind, -DT)
    g = run_gpu(ens, -200 * DT, kind, -DT)
    assert_parity(ens, g, o, sens=sens, steps=200)
    assert np.all(g["time"] == -200 * DT)
    with S.Ensemble(ens) as e:
        e.integrate(150 * DT, kind, DT)
        e.integrate(0.0, kind, -DT)
        back = e.state()
    ex, ev = per_system_errors(ens, back, ens)
    # round-off grows along the way and back like the oracle's own sensitivity
    bound = np.maximum(1e-12, 30.0 * oracle_sensitivity(ens, 150 * DT, kind, DT))
    assert np.all(ex <= bound) and np.all(ev <= bound)
    assert np.all(back["time"] == 0.0)


@pytest.mark.parametrize("kind", [O.MVS_DH, O.MVS_JACOBI])
def test_system_alone_equals_system_in_ensemble_bit_for_bit(kind):
    """Systems are handed out one by one to the groups of a warp, and a warp's last system
    runs spread over the warp's idle groups (its pair rounds and encounter tests shared
    out, gathered back in round order).  Neither changes a system's arithmetic: a system
    integrated alone (spread from its first step) equals, bit for bit, the same system
    inside an ensemble, for every body count 3..15 (single-bin launches)."""
    ens = ics.ragged(390, seed=12)
    nb = np.asarray(ens["n_body"])
    T = 300 * DT
    g = run_gpu(ens, T, kind, DT, ce=3.0, ej=100.0, single_launch=0)
    offs = np.concatenate([[0], np.cumsum(nb)])
    picked = [int(np.flatnonzero(nb == n)[k]) for n in range(3, 16) for k in (0, 5)]
    for s in picked:
        a = run_gpu(ics.subset(ens, [s]), T, kind, DT, ce=3.0, ej=100.0, single_launch=0)
        rows = slice(offs[s], offs[s + 1])
        assert a["status"][0] == g["status"][s] and a["time"][0] == g["time"][s], (s, nb[s])
        assert np.array_equal(a["pos"], g["pos"][rows]) and np.array_equal(a["vel"], g["vel"][rows]), (s, nb[s])


@pytest.mark.parametrize("kind", [O.MVS_DH, O.MVS_JACOBI])
def test_long_call_in_compacted_chunks_parity(kind):
    # 24000 steps: the call runs as 24 chunks of 1000 steps, each over the systems
    # still running, which spread over the warp's groups once they are fewer than the warps.
    # 32 tightly packed systems (9..12 mutual Hill radii, planets of 1e-7..1e-6) stop at
    # close encounters spread over the first chunks; 16 widely spaced ones (14..20 Hill
    # radii, 1e-5..1e-4) run all 1200 orbits.  Over that span two round-off histories part
    # by more than one initial 1-ulp perturbation does: each step rounds differently, and
    # the phase error of a long orbit integration grows like steps^(3/2) u (Brouwer's law,
    # ~4e-10 after 24000 steps), above the 1e-10 bar.  The survivors' states are held to
    # 30x the larger of that and the oracle's own 1-ulp sensitivity, without the 10 % cap;
    # statuses, stop times and energy errors as in every parity test.  The same call as
    # one launch agrees to the same bound (each chunk boundary stores the state in
    # barycentric coordinates and maps it back, a round-off perturbation of the survivors).
    from paper_1208_1157_gb300 import swarm as S

    ens = ics.concat(ics.mvs_compact(32, seed=17, k_lo=9.0, k_hi=12.0, m_lo=1e-7, m_hi=1e-6),
                     ics.mvs_compact(16, seed=18, k_lo=14.0, k_hi=20.0, m_lo=1e-5, m_hi=1e-4))
    T = 24000 * DT
    o = run_oracle(ens, T, kind, DT, ce=3.0, ej=100.0)
    sens = np.maximum(oracle_sensitivity(ens, T, kind, DT, ce=3.0, ej=100.0), 24000 ** 1.5 * 2.0 ** -53)
    g = run_gpu(ens, T, kind, DT, ce=3.0, ej=100.0)
    assert g["stats"]["kernel_launches"] == 2 * 24
    stop = np.round(o["time"] / DT)
    assert np.sum(o["status"] <= 1) >= 16 and np.sum((stop > 2000) & (stop < 24000)) >= 3
    assert_parity(ens, g, o, sens=sens, steps=24000, max_relaxed=1.0)
    with S.Ensemble(ens) as e:
        e.set_stop(3.0, 100.0)
        e.set_option(S.OPT_STEPS_PER_LAUNCH, 24000)
        e.integrate(T, kind, DT)
        assert e.stats()["kernel_launches"] == 2
        one = e.state()
    from gpu_util import per_system_errors
    assert np.array_equal(one["status"], g["status"]) and np.array_equal(one["time"], g["time"])
    ex, ev = per_system_errors(ens, one, g)
    assert np.all(np.maximum(ex, ev) <= np.maximum(1e-10, 30.0 * sens))


@pytest.mark.parametrize("kind", [O.MVS_DH, O.MVS_JACOBI])
def test_compacted_chunks_skip_stopped_systems_bit_for_bit(kind):
    # A 3000-step call runs as three chunks of 1000 steps, each over the bin's list
    # compacted to its runnable systems.  Systems stopped before the call (close encounter,
    # ejection) are left as they were, bit for bit; every other system ends exactly as it
    # does when the runnable systems are integrated by themselves (the hand-out and the
    # spread mode change no system's arithmetic).
    from paper_1208_1157_gb300 import swarm as S

    ens = ics.mvs_compact(200, seed=19, k_lo=6.0, k_hi=8.0)
    S_ = len(ens["n_body"])
    status = np.zeros(S_, dtype=np.int32)
    status[::7] = S.CLOSE_ENCOUNTER
    status[3::11] = S.EJECTED
    time = np.zeros(S_)
    T = 3000 * DT
    g = run_gpu(ens, T, kind, DT, ce=3.0, ej=100.0, time=time, status=status)
    assert g["stats"]["kernel_launches"] == 2 * 3
    offs = np.concatenate([[0], np.cumsum(ens["n_body"])])
    stopped = status != 0
    for s in np.flatnonzero(stopped):
        rows = slice(offs[s], offs[s + 1])
        assert g["status"][s] == status[s] and g["time"][s] == 0.0
        assert np.array_equal(g["pos"][rows], ens["pos"][rows]) and np.array_equal(g["vel"][rows], ens["vel"][rows])
    live = np.flatnonzero(~stopped)
    a = run_gpu(ics.subset(ens, live), T, kind, DT, ce=3.0, ej=100.0)
    sub = ics.subset(ens, live)
    so = np.concatenate([[0], np.cumsum(sub["n_body"])])
    for i, s in enumerate(live):
        assert a["status"][i] == g["status"][s] and a["time"][i] == g["time"][s], s
        assert np.array_equal(a["pos"][so[i]:so[i + 1]], g["pos"][offs[s]:offs[s + 1]]), s
        assert np.array_equal(a["vel"][so[i]:so[i + 1]], g["vel"][offs[s]:offs[s + 1]]), s
    assert np.sum(a["status"] >= 2) > 0 and np.sum(a["status"] == 1) > 0  # stops on the way, and survivors


@pytest.mark.parametrize("kind", [O.MVS_DH, O.MVS_JACOBI])
def test_chunked_call_keeps_log_records_in_place(kind):
    # 2500 steps with a record every 1000: the call is split into chunks of whole log
    # intervals (2000 and 500 steps here, not two of 1250), so the records fall at steps
    # 1000 and 2000 as in the oracle
    ens = ics.mvs_compact(24, seed=18, k_lo=14.0, k_hi=20.0, m_lo=1e-5, m_hi=1e-4)
    T = 2500 * DT
    o = run_oracle(ens, T, kind, DT, ce=3.0, ej=100.0, log_interval=1000, log_cap=4)
    g = run_gpu(ens, T, kind, DT, ce=3.0, ej=100.0, log_interval=1000, log_cap=4)
    assert g["stats"]["kernel_launches"] == 2 * 2
    for s in range(len(ens["n_body"])):
        lg = g["logs"][s]
        assert len(lg) == o["log_count"][s] == 2
        np.testing.assert_allclose(lg[:, 0], o["log"][s, :2, 0], rtol=1e-14)
        np.testing.assert_allclose(lg[:, 1:], o["log"][s, :2, 1:], rtol=1e-9, atol=1e-14)


@pytest.mark.parametrize("kind", [O.MVS_DH, O.MVS_JACOBI])
def test_chunked_call_with_systems_at_different_times(kind):
    # half the systems start 500 steps later than the others: the 3000-step call runs in
    # chunks sized on the longest span, the later half finishing its 2500 steps on the way;
    # against the oracle, which steps each system from its own time
    ens = ics.mvs_compact(24, seed=18, k_lo=14.0, k_hi=20.0, m_lo=1e-5, m_hi=1e-4)
    S_ = len(ens["n_body"])
    time = np.where(np.arange(S_) % 2 == 0, 0.0, 500 * DT)
    status = np.zeros(S_, dtype=np.int32)
    T = 3000 * DT
    o = run_oracle(ens, T, kind, DT, ce=3.0, ej=100.0, time=time, status=status)
    sens = np.maximum(oracle_sensitivity(ens, T, kind, DT, ce=3.0, ej=100.0, time=time, status=status),
                      3000 ** 1.5 * 2.0 ** -53)
    g = run_gpu(ens, T, kind, DT, ce=3.0, ej=100.0, time=time, status=status)
    assert g["stats"]["kernel_launches"] == 2 * 3
    assert np.all(o["status"] == 1)
    assert_parity(ens, g, o, sens=sens, steps=3000, max_relaxed=1.0)


def robust_sensitivity(ens, t_end, kind, dt, **kw):
    """The oracle's 1-ulp sensitivity taken over three perturbation patterns (positions up
    and velocities down, the reverse, and seeded random signs per element): over 10^5 steps
    one direction can happen to be nearly neutral for a system whose round-off still grows."""
    from gpu_util import per_system_errors

    base = run_oracle(ens, t_end, kind, dt, **kw)
    rs = np.random.default_rng(11)
    out = np.zeros(len(ens["n_body"]))
    for sp, sv in ((1.0, -1.0), (-1.0, 1.0), (None, None)):
        p = dict(ens)
        if sp is None:
            p["pos"] = ens["pos"] * (1 + rs.choice([-1.0, 1.0], ens["pos"].shape) * 2.0 ** -52)
            p["vel"] = ens["vel"] * (1 + rs.choice([-1.0, 1.0], ens["vel"].shape) * 2.0 ** -52)
        else:
            p["pos"] = ens["pos"] * (1 + sp * 2.0 ** -52)
            p["vel"] = ens["vel"] * (1 + sv * 2.0 ** -52)
        ex, ev = per_system_errors(ens, run_oracle(p, t_end, kind, dt, **kw), base)
        out = np.maximum(out, np.maximum(ex, ev))
    return base, out


def test_mvs_full_size_1e5_steps_sampled():
    # The 16384 x 8 Jacobi ensemble over 10^5 steps, as the benchmark runs it (auto-chunked,
    # compacted lists, spread mode for the last survivors).  Samples: 16 systems the GPU
    # leaves running and 16 it stops.  Of these, the ones whose oracle result is well
    # conditioned (1-ulp sensitivity over three perturbation patterns below 1e-6: their
    # stop step and orbit are fixed by the arithmetic, not by round-off; the chaotic rest
    # has several correct results) must match the oracle's status and time, and their
    # states within 30x the larger of that sensitivity and steps^(3/2) u (Brouwer's law).
    steps = 100000
    ens = ics.mvs_compact(16384, seed=4)
    g = run_gpu(ens, steps * DT, O.MVS_JACOBI, DT, ce=3.0, ej=100.0)
    rng = np.random.default_rng(5)
    live = np.flatnonzero(g["status"] <= 1)
    dead = np.flatnonzero(g["status"] >= 2)
    assert len(live) > 100
    idx = np.sort(np.concatenate([rng.choice(live, 16, replace=False), rng.choice(dead, 16, replace=False)]))
    sub = ics.subset(ens, idx)
    o, sens = robust_sensitivity(sub, steps * DT, O.MVS_JACOBI, DT, ce=3.0, ej=100.0)
    good = sens < 1e-6
    assert np.sum(good & (o["status"] <= 1)) >= 2 and np.sum(good & (o["status"] >= 2)) >= 8
    k = np.flatnonzero(good)
    rows = lambda d, sel: d.reshape(-1, 8, 3)[sel].reshape(-1, 3)
    gk = {"pos": rows(g["pos"], idx[k]), "vel": rows(g["vel"], idx[k]), "time": g["time"][idx[k]],
          "status": g["status"][idx[k]]}
    ok = {"pos": rows(o["pos"], k), "vel": rows(o["vel"], k), "time": o["time"][k], "status": o["status"][k]}
    bound = np.maximum(sens[k], steps ** 1.5 * 2.0 ** -53)
    assert_parity(ics.subset(sub, k), gk, ok, sens=bound, steps=steps, max_relaxed=1.0)
