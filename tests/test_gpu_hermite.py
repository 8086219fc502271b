"""GPU parity of the Hermite-4 path (C ABI -> sm_103a kernels) against the CPU oracle."""
import math

import numpy as np
import pytest

import oracle as O
from gpu_util import TWO_PI, assert_parity, block_ring_wave, oracle_sensitivity, per_system_errors, run_gpu, run_oracle
from paper_1208_1157_gb300 import ics

pytestmark = pytest.mark.gpu

DT = TWO_PI * 1e-3
MAPS = {"body_per_lane": 2, "system_per_lane": 1, "plain_per_step": 3, "auto": 0}


@pytest.fixture(scope="module")
def c1():
    # 1024 star + 2 planet systems (seed 1), 1000 steps of dt = 1e-3 inner periods
    ens = ics.three_body(1024, seed=1)
    sens = oracle_sensitivity(ens, 1000 * DT, O.HERMITE, DT, ce=3.0, ej=100.0)
    return ens, run_oracle(ens, 1000 * DT, O.HERMITE, DT, ce=3.0, ej=100.0), sens


@pytest.mark.parametrize("mapping", list(MAPS))
def test_three_body_parity_1000_steps(c1, mapping):
    ens, o, sens = c1
    g = run_gpu(ens, 1000 * DT, 1, DT, mapping=MAPS[mapping], ce=3.0, ej=100.0)
    assert_parity(ens, g, o, sens=sens, max_relaxed=0.0)  # every system on the strict 1e-10 bar
    assert g["stats"]["system_steps"] == int(np.sum(np.round(o["time"] / DT)))


def test_ragged_parity_all_body_counts():
    # n = 2..15 mixed, Hill-spaced, several warps per bin and ragged tails
    ens = ics.concat(ics.ragged(520, seed=3), ics.subset(ics.two_body(1.3, 0.2), [0]))
    o = run_oracle(ens, 200 * DT, O.HERMITE, DT, ce=3.0, ej=100.0)
    sens = oracle_sensitivity(ens, 200 * DT, O.HERMITE, DT, ce=3.0, ej=100.0)
    for single in (1, 0):
        g = run_gpu(ens, 200 * DT, 1, DT, mapping=2, ce=3.0, ej=100.0, single_launch=single)
        assert_parity(ens, g, o, sens=sens, steps=200)


def test_shortened_last_step_and_continuation():
    ens = ics.three_body(100, seed=5)
    t1 = 123.4567 * DT  # not a multiple of dt: the last step is shortened
    o = run_oracle(ens, t1, O.HERMITE, DT)
    g = run_gpu(ens, t1, 1, DT, mapping=2)
    assert_parity(ens, g, o)
    assert np.all(g["time"] == t1)
    # two calls to 2T equal one call (same steps, a0/j0 recomputed from the state)
    from paper_1208_1157_gb300 import swarm as S
    with S.Ensemble(ens) as e:
        e.integrate(300 * DT, S.HERMITE4, DT)
        e.integrate(600 * DT, S.HERMITE4, DT)
        two = e.state()
    one = run_gpu(ens, 600 * DT, 1, DT)
    ex, ev = per_system_errors(ens, two, one)
    assert ex.max() <= 1e-14 and ev.max() <= 1e-14


def test_time_reversal_on_gpu():
    ens = ics.three_body(64, seed=7)
    from paper_1208_1157_gb300 import swarm as S
    with S.Ensemble(ens) as e:
        e.set_option(S.OPT_N_CORR, 8)
        e.integrate(200 * DT, S.HERMITE4, DT)
        e.integrate(0.0, S.HERMITE4, -DT)
        back = e.state()
    ex, ev = per_system_errors(ens, back, ens)
    assert ex.max() <= 1e-13 and ev.max() <= 1e-13
    assert np.all(back["time"] == 0.0)


def test_stop_conditions_match_oracle():
    ens = ics.three_body(64, seed=8)
    # system 3: planet 2 on an escape orbit from 95 AU; system 9: planets nearly touching
    ens["pos"][3 * 3 + 2] = [95.0, 0.0, 0.0]
    ens["vel"][3 * 3 + 2] = [1.5, 0.0, 0.0]
    ens["pos"][3 * 9 + 2] = ens["pos"][3 * 9 + 1] + np.array([0.05, 0.0, 0.0])
    ens["vel"][3 * 9 + 2] = ens["vel"][3 * 9 + 1]
    o = run_oracle(ens, 3000 * DT, O.HERMITE, DT, ce=3.0, ej=100.0)
    assert o["status"][3] == O.EJECTED and o["status"][9] == O.CLOSE_ENCOUNTER
    for mapping in (2, 1, 3):
        g = run_gpu(ens, 3000 * DT, 1, DT, mapping=mapping, ce=3.0, ej=100.0)
        assert_parity(ens, g, o, check_energy=False)


def test_stopped_systems_are_not_advanced_and_zero_step_call():
    ens = ics.three_body(40, seed=9)
    st = np.zeros(40, dtype=np.int32)
    st[[1, 7]] = [O.EJECTED, O.CLOSE_ENCOUNTER]
    tm = np.zeros(40)
    o = run_oracle(ens, 50 * DT, O.HERMITE, DT, time=tm, status=st)
    g = run_gpu(ens, 50 * DT, 1, DT, time=tm, status=st)
    assert_parity(ens, g, o)
    assert np.array_equal(g["pos"][3:6], ens["pos"][3:6])
    # t_end equal to the current time: no step, status DONE, state unchanged
    g0 = run_gpu(ens, 0.0, 1, DT)
    assert np.all(g0["status"] == O.DONE) and np.array_equal(g0["pos"], ens["pos"])


def test_energy_log_matches_oracle():
    ens = ics.three_body(48, seed=10)
    o = run_oracle(ens, 1000 * DT, O.HERMITE, DT, log_interval=100, log_cap=20)
    for mapping in (2, 1, 3):
        g = run_gpu(ens, 1000 * DT, 1, DT, mapping=mapping, log_interval=100, log_cap=20)
        for s in range(48):
            lg, lo = g["logs"][s], o["log"][s, : o["log_count"][s]]
            assert lg.shape == lo.shape == (10, 5)
            np.testing.assert_allclose(lg[:, 0], lo[:, 0], rtol=1e-14)
            np.testing.assert_allclose(lg[:, 1], lo[:, 1], rtol=1e-11)
            np.testing.assert_allclose(lg[:, 2:], lo[:, 2:], rtol=1e-11, atol=1e-16)


def test_diagnostics_match_oracle():
    ens = ics.ragged(200, seed=11)
    g = run_gpu(ens, 10 * DT, 1, DT)
    offs = np.concatenate([[0], np.cumsum(ens["n_body"])])
    for s in range(200):
        sl = slice(offs[s], offs[s + 1])
        E, L = O.energy(ens["mass"][sl], g["pos"][sl], g["vel"][sl])
        assert g["energy"][s] == pytest.approx(E, rel=1e-13)
        np.testing.assert_allclose(g["angmom"][s], L, rtol=1e-12, atol=1e-18)


def test_paper_shaped_ensemble_full_size_sampled():
    # 131072 x 3 bodies, 10^4 steps: the benchmark's configuration; 32 sampled systems
    ens = ics.three_body(131072, seed=2)
    g = run_gpu(ens, 10000 * DT, 1, DT, ce=3.0, ej=100.0)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(131072, 32, replace=False))
    sub = ics.subset(ens, idx)
    o = run_oracle(sub, 10000 * DT, O.HERMITE, DT, ce=3.0, ej=100.0)
    sens = oracle_sensitivity(sub, 10000 * DT, O.HERMITE, DT, ce=3.0, ej=100.0)
    gs = {"pos": g["pos"].reshape(-1, 3, 3)[idx].reshape(-1, 3), "vel": g["vel"].reshape(-1, 3, 3)[idx].reshape(-1, 3),
          "time": g["time"][idx], "status": g["status"][idx]}
    # 10^4 steps: the 1000-step bar, scaled by the step count
    assert_parity(sub, gs, o, tol=1e-9, sens=sens, steps=10000)
    assert g["stats"]["system_steps"] > 0.99 * 131072 * 10000


@pytest.mark.parametrize("single", [0, 1])
def test_ragged_full_size_sampled(single):
    # the 65536-system ragged ensemble as the benchmark runs it (100 steps, stops on), in
    # concurrent per-bin launches (the default) and in the shared launch; 40 samples
    ens = ics.ragged(65536, seed=3)
    g = run_gpu(ens, 100 * DT, 1, DT, mapping=0, ce=3.0, ej=100.0, single_launch=single)
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(65536, 40, replace=False))
    sub = ics.subset(ens, idx)
    o = run_oracle(sub, 100 * DT, O.HERMITE, DT, ce=3.0, ej=100.0)
    sens = oracle_sensitivity(sub, 100 * DT, O.HERMITE, DT, ce=3.0, ej=100.0)
    offs = np.concatenate([[0], np.cumsum(ens["n_body"])])
    rows = np.concatenate([np.arange(offs[s], offs[s + 1]) for s in idx])
    gs = {"pos": g["pos"][rows], "vel": g["vel"][rows], "time": g["time"][idx], "status": g["status"][idx]}
    assert_parity(sub, gs, o, sens=sens, steps=100)


@pytest.mark.parametrize("mapping", [0, 3])
def test_chunked_launches_replayed_from_a_cuda_graph(mapping):
    # steps per launch = 64: the call becomes a captured graph of launches of <= 64 steps
    # (persistent), or of single steps (plain); the second call replays the same graph
    from paper_1208_1157_gb300 import swarm as S

    ens = ics.three_body(300, seed=15)
    ref = run_gpu(ens, 1000 * DT, 1, DT, mapping=mapping)
    with S.Ensemble(ens) as e:
        e.set_option(S.OPT_MAPPING, mapping)
        e.set_option(S.OPT_STEPS_PER_LAUNCH, 64)
        e.integrate(500 * DT, S.HERMITE4, DT)
        first = e.stats()["kernel_launches"]
        e.integrate(1000 * DT, S.HERMITE4, DT)
        second = e.stats()["kernel_launches"]
        got = e.state()
    assert first == second == (8 if mapping == 0 else 501)  # plain: prepare + 500 steps
    ex, ev = per_system_errors(ens, got, ref)
    assert ex.max() <= 1e-14 and ev.max() <= 1e-14
    np.testing.assert_allclose(got["time"], ref["time"], rtol=1e-14)
    assert np.all(got["status"] == O.DONE)


@pytest.mark.parametrize("mapping", [1, 2])
def test_adaptive_step_hermite_parity(mapping):
    # Eq. 5 steps with tau = 0.01 over two inner orbits, stops on
    ens = ics.three_body(200, seed=16)
    t_end = 2 * TWO_PI
    o = run_oracle(ens, t_end, O.HERMITE_ADAPTIVE, 0.01, ce=3.0, ej=100.0)
    sens = oracle_sensitivity(ens, t_end, O.HERMITE_ADAPTIVE, 0.01, ce=3.0, ej=100.0)
    g = run_gpu(ens, t_end, 4, 0.01, mapping=mapping, ce=3.0, ej=100.0)
    assert_parity(ens, g, o, sens=sens, steps=2000)
    assert np.all(g["time"][g["status"] == O.DONE] == t_end)


def test_adaptive_step_hermite_ragged_and_backwards():
    ens = ics.ragged(150, seed=17)
    t_end = 1.5 * TWO_PI
    o = run_oracle(ens, t_end, O.HERMITE_ADAPTIVE, 0.02, ce=3.0, ej=100.0)
    sens = oracle_sensitivity(ens, t_end, O.HERMITE_ADAPTIVE, 0.02, ce=3.0, ej=100.0)
    g = run_gpu(ens, t_end, 4, 0.02, ce=3.0, ej=100.0)
    assert_parity(ens, g, o, sens=sens, steps=3000)
    # a negative tau integrates back to the start time
    from paper_1208_1157_gb300 import swarm as S
    with S.Ensemble(ens) as e:
        e.integrate(t_end, S.HERMITE4_ADAPTIVE, 0.005)
        e.integrate(0.0, S.HERMITE4_ADAPTIVE, -0.005)
        back = e.state()
    assert np.all(back["time"] == 0.0)
    ex, ev = per_system_errors(ens, back, ens)
    assert np.median(np.maximum(ex, ev)) < 1e-8


@pytest.mark.parametrize("mapping", [1, 2])
def test_printed_form_corrector_parity(mapping):
    from paper_1208_1157_gb300 import swarm as S

    ens = ics.three_body(128, seed=18)
    o = O.integrate(ens, 1000 * DT, DT, O.HERMITE, corr_form=O.CORR_PRINTED, ce_factor=3.0, eject_radius=100.0)
    with S.Ensemble(ens) as e:
        e.set_option(S.OPT_MAPPING, mapping)
        e.set_option(S.OPT_CORRECTOR, 1)
        e.set_stop(3.0, 100.0)
        e.integrate(1000 * DT, S.HERMITE4, DT)
        g = e.state()
    assert_parity(ens, g, o)


def test_adaptive_full_size_sampled():
    # the paper-shaped ensemble with Eq. 5 steps (tau = 0.01) over one inner period, in the
    # benchmark's launch configuration (system per lane, systems handed out per lane)
    ens = ics.three_body(131072, seed=2)
    g = run_gpu(ens, TWO_PI, 4, 0.01, ce=3.0, ej=100.0)
    idx = np.sort(np.random.default_rng(4).choice(131072, 32, replace=False))
    sub = ics.subset(ens, idx)
    o = run_oracle(sub, TWO_PI, O.HERMITE_ADAPTIVE, 0.01, ce=3.0, ej=100.0)
    sens = oracle_sensitivity(sub, TWO_PI, O.HERMITE_ADAPTIVE, 0.01, ce=3.0, ej=100.0)
    gs = {"pos": g["pos"].reshape(-1, 3, 3)[idx].reshape(-1, 3), "vel": g["vel"].reshape(-1, 3, 3)[idx].reshape(-1, 3),
          "time": g["time"][idx], "status": g["status"][idx]}
    assert_parity(sub, gs, o, sens=sens, steps=2000)


@pytest.mark.parametrize("single", [0, 1])
def test_ragged_chunked_launches_with_forked_streams(single):
    # several body counts: per-bin launches forked onto side streams (single = 0) or the
    # shared launch next to the 16..32-body bins' launches (single = 1), captured into a
    # graph in rounds of <= 40 steps; the result equals the one-round call bit for bit
    from paper_1208_1157_gb300 import swarm as S

    ens = ics.concat(ics.ragged(260, seed=19), ics.ragged_wide(20, seed=20))
    ref = run_gpu(ens, 200 * DT, 1, DT, ce=3.0, ej=100.0, single_launch=single)
    with S.Ensemble(ens) as e:
        e.set_stop(3.0, 100.0)
        e.set_option(S.OPT_SINGLE_LAUNCH, single)
        e.set_option(S.OPT_STEPS_PER_LAUNCH, 40)
        e.integrate(200 * DT, S.HERMITE4, DT)
        launches = e.stats()["kernel_launches"]
        got = e.state()
    nbins = len(set(ens["n_body"].tolist()))
    nwide = len(set(n for n in ens["n_body"].tolist() if n >= 16))
    per_round = nbins if single == 0 else 1 + nwide
    assert launches == 5 * per_round
    assert np.array_equal(got["status"], ref["status"])
    assert np.array_equal(got["time"], ref["time"])
    assert np.array_equal(got["pos"], ref["pos"]) and np.array_equal(got["vel"], ref["vel"])


def test_chunked_graph_is_recaptured_when_the_corrector_changes():
    # same step count per call, corrector switched between calls: the replayed graph must
    # not keep the first call's corrector
    from paper_1208_1157_gb300 import swarm as S

    ens = ics.three_body(64, seed=21)
    with S.Ensemble(ens) as e:
        e.set_option(S.OPT_CORRECTOR, 1)
        e.integrate(300 * DT, S.HERMITE4, DT)
        ref = e.state()
    with S.Ensemble(ens) as e:
        e.set_option(S.OPT_STEPS_PER_LAUNCH, 50)
        e.integrate(300 * DT, S.HERMITE4, DT)  # time-symmetric corrector, captured
        e.set_state(ens["pos"], ens["vel"], time=[0.0] * 64, status=[0] * 64)
        e.set_option(S.OPT_CORRECTOR, 1)
        e.integrate(300 * DT, S.HERMITE4, DT)  # same shape of call, printed corrector
        got = e.state()
    assert np.array_equal(got["pos"], ref["pos"]) and np.array_equal(got["vel"], ref["vel"])


def test_device_pointer_state_round_trip():
    # state in and out through device arrays (torch tensors on the ensemble's stream)
    import torch
    from paper_1208_1157_gb300 import swarm as S

    ens = ics.ragged(200, seed=22)
    ref = run_gpu(ens, 100 * DT, 1, DT)
    nb, ns = int(np.sum(ens["n_body"])), len(ens["n_body"])
    stream = torch.cuda.current_stream()
    with S.Ensemble(ens, stream=stream) as e:
        e.integrate(37 * DT, S.HERMITE4, DT)  # move away from the initial state
        pos_t = torch.tensor(ens["pos"], dtype=torch.float64, device="cuda")
        vel_t = torch.tensor(ens["vel"], dtype=torch.float64, device="cuda")
        time_t = torch.zeros(ns, dtype=torch.float64, device="cuda")
        st_t = torch.zeros(ns, dtype=torch.int32, device="cuda")
        e.set_state_dev(pos_t, vel_t, time_t, st_t)
        e.integrate(100 * DT, S.HERMITE4, DT)
        out_p = torch.empty((nb, 3), dtype=torch.float64, device="cuda")
        out_v = torch.empty((nb, 3), dtype=torch.float64, device="cuda")
        out_t = torch.empty(ns, dtype=torch.float64, device="cuda")
        out_s = torch.empty(ns, dtype=torch.int32, device="cuda")
        e.state_dev(out_p, out_v, out_t, out_s)
        stream.synchronize()
    assert np.array_equal(out_p.cpu().numpy(), ref["pos"]) and np.array_equal(out_v.cpu().numpy(), ref["vel"])
    assert np.array_equal(out_t.cpu().numpy(), ref["time"]) and np.array_equal(out_s.cpu().numpy(), ref["status"])


def test_checkpoint_and_resume(tmp_path):
    # stop half way, write the state to disk, resume in a new ensemble: the same states
    # as one call, bit for bit (a0, j0 are recomputed from the stored state)
    from paper_1208_1157_gb300 import swarm as S

    ens = ics.ragged(150, seed=23)
    ref = run_gpu(ens, 400 * DT, 1, DT, ce=3.0, ej=100.0)
    with S.Ensemble(ens) as e:
        e.set_stop(3.0, 100.0)
        e.integrate(150 * DT, S.HERMITE4, DT)
        S.save_checkpoint(e, str(tmp_path / "ck.npz"))
    with S.resume(S.load_checkpoint(str(tmp_path / "ck.npz"))) as e:
        e.set_stop(3.0, 100.0)
        e.integrate(400 * DT, S.HERMITE4, DT)
        got = e.state()
    for k in ("pos", "vel", "status"):
        assert np.array_equal(got[k], ref[k]), k
    # times are t0 + k dt from each call's start, so a stop time after the resume can
    # differ from the one-call value in the last place
    np.testing.assert_allclose(got["time"], ref["time"], rtol=1e-15, atol=0)


def _hierarchical_triples(k, seed):
    """k triples of comparable masses: an inner binary (separation 1, circular) and a
    third body on a circular orbit of radius 8 about it, random phases and planes."""
    rng = np.random.default_rng(seed)
    mass, pos, vel = [], [], []
    for _ in range(k):
        m = rng.uniform(0.3, 1.0, 3)
        mb = m[0] + m[1]
        ph, ph3 = rng.uniform(0, 2 * np.pi, 2)
        r1 = np.array([np.cos(ph), np.sin(ph), 0.0])
        v1 = np.sqrt(mb) * np.array([-np.sin(ph), np.cos(ph), 0.0])
        x = [-m[1] / mb * r1, m[0] / mb * r1]
        v = [-m[1] / mb * v1, m[0] / mb * v1]
        R = 8.0 * np.array([np.cos(ph3), np.sin(ph3), 0.0])
        V = np.sqrt((mb + m[2]) / 8.0) * np.array([-np.sin(ph3), np.cos(ph3), 0.0])
        M = mb + m[2]
        X = [xi - m[2] / M * R for xi in x] + [mb / M * R]
        U = [vi - m[2] / M * V for vi in v] + [mb / M * V]
        # random plane of the whole configuration
        a, b = rng.uniform(0, np.pi, 2)
        rot = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]]) @ \
            np.array([[1, 0, 0], [0, np.cos(b), -np.sin(b)], [0, np.sin(b), np.cos(b)]])
        mass += list(m)
        pos += [rot @ p for p in X]
        vel += [rot @ u for u in U]
    return {"n_body": np.full(k, 3, dtype=np.int32), "mass": np.array(mass), "pos": np.array(pos),
            "vel": np.array(vel)}


@pytest.mark.parametrize("integrator", [1, 5])
def test_comparable_masses_parity(integrator):
    # the system-per-lane kernels step coordinates relative to body 0; with no dominant
    # body that frame is no better conditioned than the inertial one and must still agree
    ens = _hierarchical_triples(64, seed=29)
    dt = 2 * math.pi * 1e-3
    o = run_oracle(ens, 500 * dt, integrator, dt)
    sens = oracle_sensitivity(ens, 500 * dt, integrator, dt)
    g = run_gpu(ens, 500 * dt, integrator, dt)
    assert_parity(ens, g, o, sens=sens, steps=500)


@pytest.mark.parametrize("ns", [(7, 9), (13, 14)])
def test_block_ring_equals_warp_ring_bit_for_bit(ns):
    # Bins large enough for the CTA-packed body-per-lane kernel (one wave of its CTAs),
    # integrated by single-bin launches (packed over the CTA, shared-memory exchange) and by
    # the shared multi-bin launch (warp ring, shuffles): the same bits, energy logs included.
    from paper_1208_1157_gb300 import swarm as S

    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    parts = [ics.request_ensemble({"n_sys": block_ring_wave(n, sms) + 37, "n": n, "seed": 600 + n}) for n in ns]
    ens = ics.concat(*parts)
    a = run_gpu(ens, 60 * DT, 1, DT, mapping=S.MAP_BODY_PER_LANE, ce=3.0, ej=100.0, single_launch=0,
                log_interval=20, log_cap=4)
    b = run_gpu(ens, 60 * DT, 1, DT, mapping=S.MAP_BODY_PER_LANE, ce=3.0, ej=100.0, single_launch=1,
                log_interval=20, log_cap=4)
    for k in ("pos", "vel", "time", "status"):
        assert np.array_equal(a[k], b[k]), k
    assert all(np.array_equal(x, y) for x, y in zip(a["logs"], b["logs"]))
