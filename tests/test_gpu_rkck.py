"""GPU parity of the Runge-Kutta Cash-Karp path (Sec. 2.2.2, Sec. 4.3.3; C ABI -> sm_103a
kernels) against the CPU oracle."""
import numpy as np
import pytest

import oracle as O
from gpu_util import TWO_PI, assert_parity, block_ring_wave, oracle_sensitivity, per_system_errors, run_gpu, run_oracle
from paper_1208_1157_gb300 import ics

pytestmark = pytest.mark.gpu

DT = TWO_PI * 1e-3
RKCK, RKCK_ADAPTIVE = 5, 6


def pairs(ens):
    n = np.asarray(ens["n_body"], dtype=np.int64)
    return n * (n - 1) // 2


def test_rkck_fixed_three_body_parity_and_counters():
    ens = ics.three_body(512, seed=21)
    t_end = 1000 * DT
    o = run_oracle(ens, t_end, O.RKCK, DT, ce=3.0, ej=100.0)
    sens = oracle_sensitivity(ens, t_end, O.RKCK, DT, ce=3.0, ej=100.0)
    g = run_gpu(ens, t_end, RKCK, DT, ce=3.0, ej=100.0)
    assert_parity(ens, g, o, sens=sens)
    steps = np.round(o["time"] / DT).astype(np.int64)
    assert g["stats"]["system_steps"] == int(steps.sum())
    # six force evaluations per step plus the first stage of the first step
    assert g["stats"]["pair_evaluations"] == int(np.sum(pairs(ens) * (1 + 6 * steps)))


def test_rkck_fixed_ragged_parity_with_a_shortened_last_step():
    # n = 2..15 with ragged tails; t_end not a multiple of dt
    ens = ics.concat(ics.ragged(300, seed=22), ics.subset(ics.two_body(1.2, 0.3), [0]))
    t_end = 150.37 * DT
    o = run_oracle(ens, t_end, O.RKCK, DT, ce=3.0, ej=100.0)
    sens = oracle_sensitivity(ens, t_end, O.RKCK, DT, ce=3.0, ej=100.0)
    g = run_gpu(ens, t_end, RKCK, DT, ce=3.0, ej=100.0)
    assert_parity(ens, g, o, sens=sens, steps=151)
    assert np.all(g["time"][g["status"] == O.DONE] == t_end)


def test_rkck_adaptive_three_body_parity():
    ens = ics.three_body(256, seed=23)
    t_end = TWO_PI
    kw = dict(ce=3.0, ej=100.0, rk_eps=1e-10)
    o = run_oracle(ens, t_end, O.RKCK_ADAPTIVE, 0.05, log_interval=1, log_cap=2000, **kw)
    sens = oracle_sensitivity(ens, t_end, O.RKCK_ADAPTIVE, 0.05, **kw)
    g = run_gpu(ens, t_end, RKCK_ADAPTIVE, 0.05, **kw)
    assert_parity(ens, g, o, sens=sens, steps=int(o["log_count"].max()), stop_time_rtol=1e-8)
    assert np.all(g["time"][g["status"] == O.DONE] == t_end)
    # the same accepted steps (one log record per accepted step in the oracle run)
    assert g["stats"]["system_steps"] == int(o["log_count"].sum())


def test_rkck_adaptive_ragged_rejections_and_backwards():
    # a first trial of many orbits is rejected until the error estimate is met
    ens = ics.ragged(120, seed=24)
    t_end = TWO_PI
    kw = dict(ce=3.0, ej=100.0, rk_eps=1e-11)
    o = run_oracle(ens, t_end, O.RKCK_ADAPTIVE, 5.0, **kw)
    sens = oracle_sensitivity(ens, t_end, O.RKCK_ADAPTIVE, 5.0, **kw)
    g = run_gpu(ens, t_end, RKCK_ADAPTIVE, 5.0, **kw)
    assert_parity(ens, g, o, sens=sens, steps=5000, stop_time_rtol=1e-8)
    from paper_1208_1157_gb300 import swarm as S
    with S.Ensemble(ens) as e:
        e.set_tolerance(1e-12)
        e.integrate(t_end, S.RKCK_ADAPTIVE, 0.01)
        e.integrate(0.0, S.RKCK_ADAPTIVE, -0.01)
        back = e.state()
    assert np.all(back["time"] == 0.0)
    ex, ev = per_system_errors(ens, back, ens)
    assert np.median(np.maximum(ex, ev)) < 1e-8


def test_rkck_chunked_graph_launches_equal_one_launch():
    ens = ics.three_body(96, seed=25)
    one = run_gpu(ens, 1000 * DT, RKCK, DT)
    chunked = run_gpu(ens, 1000 * DT, RKCK, DT, steps_per_launch=100)
    assert chunked["stats"]["kernel_launches"] == 10
    ex, ev = per_system_errors(ens, chunked, one)
    # every launch boundary rounds the state once through inertial coordinates (the
    # 3-body kernel steps coordinates relative to body 0): agreement to round-off
    assert ex.max() <= 1e-14 and ev.max() <= 1e-14


def test_rkck_tolerance_is_checked():
    from paper_1208_1157_gb300 import swarm as S
    with S.Ensemble(ics.three_body(4, seed=1)) as e:
        for bad in (0.0, -1e-9, 1.0, float("nan")):
            with pytest.raises(S.SwarmError):
                e.set_tolerance(bad)


def sample_rows(ens, g, idx):
    n = int(ens["n_body"][0])
    return {"pos": g["pos"].reshape(-1, n, 3)[idx].reshape(-1, 3), "vel": g["vel"].reshape(-1, n, 3)[idx].reshape(-1, 3),
            "time": g["time"][idx], "status": g["status"][idx]}


def test_rkck_full_size_sampled():
    # the paper-shaped ensemble (131072 x 3) in the benchmark's launch configuration:
    # 500 fixed steps and one inner period of adaptive steps, 32 sampled systems each
    ens = ics.three_body(131072, seed=2)
    idx = np.sort(np.random.default_rng(3).choice(131072, 32, replace=False))
    sub = ics.subset(ens, idx)
    g = run_gpu(ens, 500 * DT, RKCK, DT, ce=3.0, ej=100.0)
    o = run_oracle(sub, 500 * DT, O.RKCK, DT, ce=3.0, ej=100.0)
    assert_parity(sub, sample_rows(ens, g, idx), o, sens=oracle_sensitivity(sub, 500 * DT, O.RKCK, DT, ce=3.0, ej=100.0),
                  steps=500)
    g = run_gpu(ens, TWO_PI, RKCK_ADAPTIVE, 0.05, ce=3.0, ej=100.0)
    o = run_oracle(sub, TWO_PI, O.RKCK_ADAPTIVE, 0.05, ce=3.0, ej=100.0)
    sens = oracle_sensitivity(sub, TWO_PI, O.RKCK_ADAPTIVE, 0.05, ce=3.0, ej=100.0)
    assert_parity(sub, sample_rows(ens, g, idx), o, sens=sens, steps=1000, stop_time_rtol=1e-8)


def test_rkck_fixed_backward_parity():
    # negative fixed steps, ragged n with a shortened last step
    ens = ics.ragged(200, seed=27)
    t_end = -120.6 * DT
    o = run_oracle(ens, t_end, O.RKCK, -DT, ce=3.0, ej=100.0)
    sens = oracle_sensitivity(ens, t_end, O.RKCK, -DT, ce=3.0, ej=100.0)
    g = run_gpu(ens, t_end, RKCK, -DT, ce=3.0, ej=100.0)
    assert_parity(ens, g, o, sens=sens, steps=121)


@pytest.mark.parametrize("ns", [(7, 9), (13, 14)])
def test_block_ring_equals_warp_ring_bit_for_bit(ns):
    # Bins large enough for the CTA-packed body-per-lane kernel (one wave of its CTAs)
    # against 40 of their systems integrated alone (small bins: the warp ring): the same bits.
    from paper_1208_1157_gb300 import swarm as S

    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    parts = [ics.request_ensemble({"n_sys": block_ring_wave(n, sms) + 37, "n": n, "seed": 700 + n}) for n in ns]
    ens = ics.concat(*parts)
    a = run_gpu(ens, 40 * DT, S.RKCK, DT, ce=3.0, ej=100.0)
    nb = np.asarray(ens["n_body"])
    offs = np.concatenate([[0], np.cumsum(nb)])
    idx = np.sort(np.random.default_rng(3).choice(len(nb), 40, replace=False))
    b = run_gpu(ics.subset(ens, idx), 40 * DT, S.RKCK, DT, ce=3.0, ej=100.0)
    rows = np.concatenate([np.arange(offs[s], offs[s + 1]) for s in idx])
    assert np.array_equal(a["pos"][rows], b["pos"]) and np.array_equal(a["vel"][rows], b["vel"])
    assert np.array_equal(a["time"][idx], b["time"]) and np.array_equal(a["status"][idx], b["status"])
