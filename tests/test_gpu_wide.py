"""GPU parity of the Hermite path for larger systems (16..32 bodies, one system per warp)
against the CPU oracle, alone and mixed with the per-n bins."""
import numpy as np
import pytest

import oracle as O
from gpu_util import TWO_PI, assert_parity, oracle_sensitivity, per_system_errors, run_gpu, run_oracle
from paper_1208_1157_gb300 import ics

pytestmark = pytest.mark.gpu

DT = TWO_PI * 1e-3


@pytest.fixture(scope="module")
def wide():
    ens = ics.ragged_wide(160, seed=31)  # n = 16..32, several systems of every count
    t_end = 200 * DT
    o = run_oracle(ens, t_end, O.HERMITE, DT, ce=3.0, ej=100.0)
    sens = oracle_sensitivity(ens, t_end, O.HERMITE, DT, ce=3.0, ej=100.0)
    return ens, t_end, o, sens


def test_wide_hermite_parity(wide):
    ens, t_end, o, sens = wide
    g = run_gpu(ens, t_end, 1, DT, ce=3.0, ej=100.0)
    assert_parity(ens, g, o, sens=sens, steps=200)
    n = ens["n_body"].astype(np.int64)
    steps = np.round(o["time"] / DT).astype(np.int64)
    assert g["stats"]["system_steps"] == int(steps.sum())
    assert g["stats"]["pair_evaluations"] == int(np.sum(n * (n - 1) // 2 * (1 + 3 * steps)))


def test_wide_and_small_bins_in_one_call():
    # the per-n bins share one launch (or get one each) next to the wide bins' launch
    ens = ics.concat(ics.ragged(200, seed=32), ics.ragged_wide(60, seed=33))
    t_end = 120.5 * DT  # shortened last step
    o = run_oracle(ens, t_end, O.HERMITE, DT, ce=3.0, ej=100.0)
    sens = oracle_sensitivity(ens, t_end, O.HERMITE, DT, ce=3.0, ej=100.0)
    for single in (1, 0):
        g = run_gpu(ens, t_end, 1, DT, ce=3.0, ej=100.0, single_launch=single)
        assert_parity(ens, g, o, sens=sens, steps=121)


def test_wide_adaptive_and_printed_corrector():
    ens = ics.ragged_wide(48, seed=34)
    t_end = 0.5 * TWO_PI
    o = run_oracle(ens, t_end, O.HERMITE_ADAPTIVE, 0.01, ce=3.0, ej=100.0)
    sens = oracle_sensitivity(ens, t_end, O.HERMITE_ADAPTIVE, 0.01, ce=3.0, ej=100.0)
    g = run_gpu(ens, t_end, 4, 0.01, ce=3.0, ej=100.0)
    assert_parity(ens, g, o, sens=sens, steps=5000)
    from paper_1208_1157_gb300 import swarm as S
    o2 = O.integrate(ens, 100 * DT, DT, O.HERMITE, corr_form=O.CORR_PRINTED)
    with S.Ensemble(ens) as e:
        e.set_option(S.OPT_CORRECTOR, 1)
        e.integrate(100 * DT, S.HERMITE4, DT)
        g2 = e.state()
    assert_parity(ens, g2, o2, steps=100)


def test_wide_logs_and_chunked_launches():
    ens = ics.ragged_wide(40, seed=35, n_min=21, n_max=21)  # one bin: one launch per chunk
    o = run_oracle(ens, 300 * DT, O.HERMITE, DT, log_interval=100, log_cap=8)
    g = run_gpu(ens, 300 * DT, 1, DT, log_interval=100, log_cap=8)
    for s in range(len(ens["n_body"])):
        lg = g["logs"][s]
        assert len(lg) == 3
        np.testing.assert_allclose(lg[:, 0], o["log"][s, :3, 0], rtol=1e-14)
        np.testing.assert_allclose(lg[:, 1:], o["log"][s, :3, 1:], rtol=1e-10, atol=1e-14)
    one = run_gpu(ens, 300 * DT, 1, DT)
    chunked = run_gpu(ens, 300 * DT, 1, DT, steps_per_launch=64)
    assert chunked["stats"]["kernel_launches"] == 5
    ex, ev = per_system_errors(ens, chunked, one)
    assert ex.max() == 0.0 and ev.max() == 0.0


@pytest.mark.parametrize("kind", [O.MVS_DH, O.MVS_JACOBI])
def test_wide_mvs_parity(kind):
    # 16..32-body systems next to smaller ones, dt = 1/20 inner period, shortened last
    # step, stops on (2 mutual Hill radii: the stops spread over the call), logs every 50
    # steps
    ens = ics.concat(ics.ragged_wide(48, seed=36), ics.ragged(40, seed=39, n_max=8))
    dt = TWO_PI / 20
    t_end = 300.5 * dt
    o = run_oracle(ens, t_end, kind, dt, ce=2.0, ej=100.0, log_interval=50, log_cap=8)
    sens = oracle_sensitivity(ens, t_end, kind, dt, ce=2.0, ej=100.0)
    g = run_gpu(ens, t_end, kind, dt, ce=2.0, ej=100.0, log_interval=50, log_cap=8)
    assert_parity(ens, g, o, sens=sens, steps=301)
    for s in range(len(ens["n_body"])):
        lg = g["logs"][s]
        assert len(lg) == o["log_count"][s]
        if len(lg):
            np.testing.assert_allclose(lg[:, 0], o["log"][s, :len(lg), 0], rtol=1e-14)


def test_wide_runge_kutta_parity():
    # fixed steps (shortened last one) and adaptive steps on 16..32-body systems, mixed
    # with smaller ones in the same ensemble
    ens = ics.concat(ics.ragged_wide(48, seed=37), ics.ragged(40, seed=38))
    t_end = 80.5 * DT
    o = run_oracle(ens, t_end, O.RKCK, DT, ce=3.0, ej=100.0)
    sens = oracle_sensitivity(ens, t_end, O.RKCK, DT, ce=3.0, ej=100.0)
    g = run_gpu(ens, t_end, 5, DT, ce=3.0, ej=100.0)
    assert_parity(ens, g, o, sens=sens, steps=81)
    kw = dict(ce=3.0, ej=100.0, rk_eps=1e-11)
    o = run_oracle(ens, 0.3 * TWO_PI, O.RKCK_ADAPTIVE, 0.05, **kw)
    sens = oracle_sensitivity(ens, 0.3 * TWO_PI, O.RKCK_ADAPTIVE, 0.05, **kw)
    g = run_gpu(ens, 0.3 * TWO_PI, 6, 0.05, **kw)
    assert_parity(ens, g, o, sens=sens, steps=2000, stop_time_rtol=1e-8)


def test_wide_full_size_sampled():
    # the 16384-system 16..32-body ensemble of the benchmark, 20 steps, 24 sampled systems
    ens = ics.ragged_wide(16384, seed=6)
    g = run_gpu(ens, 20 * DT, 1, DT, ce=3.0, ej=100.0)
    idx = np.sort(np.random.default_rng(5).choice(16384, 24, replace=False))
    sub = ics.subset(ens, idx)
    o = run_oracle(sub, 20 * DT, O.HERMITE, DT, ce=3.0, ej=100.0)
    offs = np.concatenate([[0], np.cumsum(ens["n_body"])])
    rows = np.concatenate([np.arange(offs[i], offs[i + 1]) for i in idx])
    gs = {"pos": g["pos"][rows], "vel": g["vel"][rows], "time": g["time"][idx], "status": g["status"][idx]}
    assert_parity(sub, gs, o, steps=20)
