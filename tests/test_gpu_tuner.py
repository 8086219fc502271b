"""The autotuner (swarm_tuner_choice) against its own candidates timed directly on the
same shape, and an automatically mapped ensemble against a fixed mapping."""
import math

import numpy as np
import pytest

from gpu_util import per_system_errors
from paper_1208_1157_gb300 import ics

pytestmark = pytest.mark.gpu

HDT = 2 * math.pi * 1e-3
MDT = 2 * math.pi / 20


def shape_ensemble(n, integ, n_sys):
    if integ == 3:  # the compact 8-body MVS ensemble
        return ics.mvs_compact(n_sys, seed=4, n=n)
    return ics.request_ensemble({"n_sys": n_sys, "n": n, "seed": 77})


def candidates(n, integ):
    # the tuner's candidate list (csrc/tuner.cu, tuner_candidates): body per lane at full
    # residency and 1, 2, 3 CTAs per SM; a system per lane for small Hermite systems
    c = [(2, 0), (2, 1), (2, 2), (2, 3)]
    if integ == 1 and n <= 4:
        c += [(1, 0), (1, 1)] + ([(1, 3)] if n <= 3 else [])
    return c


def rate(ens, integ, mapping, ctas, steps=64):
    from paper_1208_1157_gb300 import swarm as S

    dt = HDT if integ == 1 else MDT
    best = 0.0
    with S.Ensemble(ens) as e:
        e.set_option(S.OPT_MAPPING, mapping)
        e.set_option(S.OPT_CTAS_PER_SM, ctas)
        for rep in range(4):  # the first call warms up
            e.integrate((rep + 1) * steps * dt, integ, dt)
            st = e.stats()
            if rep:
                best = max(best, st["system_steps"] / (st["kernel_ms"] * 1e-3))
    return best


@pytest.mark.parametrize("n,integ,n_sys", [(8, 3, 16384), (13, 1, 5041)])
def test_tuner_choice_within_5_percent_of_the_best_candidate(n, integ, n_sys):
    from paper_1208_1157_gb300 import swarm as S

    m, c = S.tuner_choice(n, integ, n_sys)
    cands = candidates(n, integ)
    assert (m, c) in cands
    ens = shape_ensemble(n, integ, n_sys)
    rates = {cd: rate(ens, integ, *cd) for cd in cands}
    best = max(rates.values())
    print(f"n={n} integrator={integ}: choice {(m, c)} at {rates[(m, c)]:.3e}, best {best:.3e}; "
          + ", ".join(f"{k}: {v:.3e}" for k, v in rates.items()))
    assert rates[(m, c)] >= 0.95 * best, rates


@pytest.mark.parametrize("n,integ,n_sys", [(8, 3, 16384), (13, 1, 5041)])
def test_tuned_mapping_gives_the_fixed_mappings_results(n, integ, n_sys):
    from paper_1208_1157_gb300 import swarm as S

    ens = shape_ensemble(n, integ, n_sys)
    dt = HDT if integ == 1 else MDT
    out = {}
    for mapping in (S.MAP_AUTO, S.MAP_BODY_PER_LANE):
        with S.Ensemble(ens) as e:
            e.set_option(S.OPT_MAPPING, mapping)
            e.set_stop(3.0, 100.0)
            e.integrate(300 * dt, integ, dt)
            out[mapping] = e.state()
    a, b = out[S.MAP_AUTO], out[S.MAP_BODY_PER_LANE]
    assert np.array_equal(a["status"], b["status"]) and np.array_equal(a["time"], b["time"])
    ex, ev = per_system_errors(ens, a, b)
    assert ex.max() <= 1e-10 and ev.max() <= 1e-10
