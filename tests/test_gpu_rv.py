"""Radial-velocity observable (on-device reduction to one number per system and
observation) against the CPU oracle."""
import math

import numpy as np
import pytest

import oracle as O
from gpu_util import TWO_PI
from paper_1208_1157_gb300 import ics

pytestmark = pytest.mark.gpu

DT = TWO_PI * 1e-3
LOS = (0.6, 0.0, 0.8)


def speed_scale(ens):
    offs = np.concatenate([[0], np.cumsum(ens["n_body"])])
    return np.array([np.abs(ens["vel"][offs[s]:offs[s + 1]]).max() for s in range(len(ens["n_body"]))])


@pytest.mark.parametrize("integ,dt", [(1, DT), (6, 0.02), (3, TWO_PI / 20)])
def test_observed_radial_velocities_match_the_oracle(integ, dt):
    from paper_1208_1157_gb300 import swarm as S

    ens = ics.ragged(200, seed=41, n_max=8)
    t_obs = np.sort(np.concatenate([[0.0], 0.37 + 3.0 * np.arange(11) / 11.0 * TWO_PI / 3]))
    o = O.observe_rv(ens, t_obs, dt, integ, los=LOS, ce_factor=3.0, eject_radius=100.0)
    with S.Ensemble(ens) as e:
        e.set_stop(3.0, 100.0)
        rv = e.observe_rv(t_obs, integ, dt, los=LOS)
        st = e.state()
    assert np.array_equal(st["status"], o["status"])
    err = np.abs(rv - o["rv"]).max(axis=0) / speed_scale(ens)
    assert np.median(err) < 1e-12 and err.max() < 1e-9, (np.median(err), err.max())


def test_query_rv_is_the_central_body_velocity_along_the_line_of_sight():
    from paper_1208_1157_gb300 import swarm as S

    ens = ics.three_body(333, seed=42)
    with S.Ensemble(ens) as e:
        e.integrate(50 * DT, S.HERMITE4, DT)
        rv = e.rv(LOS)
        st = e.state()
    v0 = st["vel"][0::3]
    want = v0 @ np.array(LOS)
    assert np.abs(rv - want).max() <= 1e-18 + 1e-15 * np.abs(want).max()


def test_rv_arguments_are_checked():
    from paper_1208_1157_gb300 import swarm as S

    with S.Ensemble(ics.three_body(8, seed=43)) as e:
        with pytest.raises(S.SwarmError):
            e.rv((1.0, 1.0, 0.0))  # not a unit vector
        with pytest.raises(S.SwarmError):
            e.observe_rv([1.0, 0.5], S.HERMITE4, DT)  # times run against dt
        back = e.observe_rv([0.0, -0.5, -1.0], S.HERMITE4, -DT)
        assert back.shape == (3, 8) and np.all(np.isfinite(back))
