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


def test_wide_systems_refuse_the_other_integrators():
    from paper_1208_1157_gb300 import swarm as S
    with S.Ensemble(ics.ragged_wide(4, seed=36)) as e:
        for integ in (S.MVS_DH, S.MVS_JACOBI, S.RKCK, S.RKCK_ADAPTIVE):
            with pytest.raises(S.SwarmError):
                e.integrate(0.1, integ, 0.01)
