"""Continuous batching: requests served in a mix give the same results as alone, and
the oracle's; systems retire one by one and their slots are backfilled at once."""
import math

import numpy as np
import pytest

from gpu_util import assert_parity, oracle_sensitivity, per_system_errors, run_oracle
from paper_1208_1157_gb300 import ics

pytestmark = pytest.mark.gpu

HDT = 2 * math.pi * 1e-3
MDT = 2 * math.pi / 20
INTEG = {1: 1, 2: 2, 3: 3}


def small_trace(seed=31, k=14):
    rng = np.random.default_rng(seed)
    trace = []
    for r in range(k):
        integ = int(rng.integers(1, 4))
        n = int(rng.choice([3, 5, 8, 13]))
        steps = int(rng.integers(20, 260)) if integ == 1 else int(rng.integers(10, 90))
        dt = HDT if integ == 1 else MDT
        trace.append({"id": r, "arrival_s": 0.004 * r, "n_sys": int(rng.integers(1, 150)), "n": n,
                      "integrator": integ, "t_end": (steps + 0.37) * dt, "seed": 1000 + r})
    return trace


def alone(ens, t_end, integ, ce=3.0, ej=100.0):
    from paper_1208_1157_gb300 import swarm as S

    with S.Ensemble(ens) as e:
        e.set_stop(ce, ej)
        e.integrate(t_end, integ, HDT if integ == 1 else MDT)
        return e.state()


def check_same(trace, ens_list, out, tol=1e-10):
    """Each served result equals the same request run alone through an ensemble (1e-10)
    and matches the oracle under the parity criteria of every other GPU test."""
    for r, q in enumerate(trace):
        res = out["done"][r]
        ref = alone(ens_list[r], q["t_end"], q["integrator"])
        assert np.array_equal(res["status"], ref["status"]), f"request {r}"
        np.testing.assert_allclose(res["time"], ref["time"], rtol=1e-13, atol=0)
        ex, ev = per_system_errors(ens_list[r], res, ref)
        assert ex.max() <= tol and ev.max() <= tol, (r, ex.max(), ev.max())
        dt = HDT if q["integrator"] == 1 else MDT
        kw = dict(ce=3.0, ej=100.0)
        o = run_oracle(ens_list[r], q["t_end"], q["integrator"], dt, **kw)
        sens = oracle_sensitivity(ens_list[r], q["t_end"], q["integrator"], dt, **kw)
        assert_parity(ens_list[r], res, o, sens=sens, steps=int(math.ceil(q["t_end"] / dt)))


def test_results_in_the_mix_equal_results_alone():
    from paper_1208_1157_gb300 import server as SV

    trace = small_trace()
    ens_list = [ics.request_ensemble(q) for q in trace]
    with SV.Server(slots_per_pool=512, quantum_steps=37) as sv:
        out = SV.replay(sv, trace, ens_list, collect=True)
        st = sv.stats()
    assert st["completed"] == len(trace) and st["queued"] == 0
    assert st["quanta"] > 1
    check_same(trace, ens_list, out)


def test_backfill_when_pools_are_full():
    # pools of 64 slots: the 5-body Hermite requests below need 150 slots in total; the
    # first round fills every slot (request 0 whole, 14 systems of request 1), the rest
    # waits in arrival order until systems retire and free their slots
    from paper_1208_1157_gb300 import server as SV

    trace = [{"id": r, "arrival_s": 0.0, "n_sys": 50, "n": 5, "integrator": 1, "t_end": (40 + 30 * r) * HDT,
              "seed": 2000 + r} for r in range(3)]
    ens_list = [ics.request_ensemble(q) for q in trace]
    with SV.Server(slots_per_pool=64, quantum_steps=25) as sv:
        for q, e in zip(trace, ens_list):
            sv.submit(e, q["t_end"], 1)
        sv.step()
        st = sv.stats()
        # every slot was filled; the systems that stopped within the first quantum (the
        # oracle's count) have retired already
        first = ics.concat(ens_list[0], ics.subset(ens_list[1], range(14)))
        early = int(np.sum(run_oracle(first, 25 * HDT, 1, HDT, ce=3.0, ej=100.0)["status"] >= 2))
        assert st["admitted"] == 2 and st["queued"] == 2 and st["occupied_slots"] == 64 - early
        assert sv.poll(3)[0] == SV.REQ_QUEUED  # request 2 waits behind request 1
        out = {"done": {}}
        for _ in range(200):
            sv.step()
            if sv.stats()["completed"] == 3:
                break
        for r, q in enumerate(trace):
            state, res = sv.poll(r + 1, q["n_sys"], q["n"])
            assert state == SV.REQ_DONE
            out["done"][r] = res
    check_same(trace, ens_list, out)


def test_memory_budget_releases_idle_pools():
    from paper_1208_1157_gb300 import server as SV

    trace = [{"id": r, "arrival_s": 0.0, "n_sys": 20, "n": n, "integrator": 1, "t_end": 30 * HDT, "seed": 3000 + r}
             for r, n in enumerate([3, 4, 6, 7])]
    ens_list = [ics.request_ensemble(q) for q in trace]
    one_pool = 32 * (7 * 7 + 2) * 8 + 3 * 4 * 32 + 4  # the largest of these pools (n = 7, 32 slots)
    with SV.Server(slots_per_pool=32, quantum_steps=10, device_bytes=one_pool) as sv:
        out = SV.replay(sv, trace, ens_list, collect=True)
        st = sv.stats()
    assert st["completed"] == 4 and st["device_bytes"] <= one_pool
    check_same(trace, ens_list, out)


def test_stopped_systems_retire_at_once_and_their_slots_are_backfilled():
    # Pool of 64 slots.  Request A: 40 systems, 12 of them with a planet placed to be
    # ejected within the first quantum; request B: 36 systems, of which 24 fit at first.
    # After the first round the 12 ejected systems of A retire alone, and the next round
    # admits B's remaining 12 systems into their slots while A is still running.
    from paper_1208_1157_gb300 import server as SV

    qa = {"id": 0, "arrival_s": 0.0, "n_sys": 40, "n": 3, "integrator": 1, "t_end": 300 * HDT, "seed": 0}
    qb = {"id": 1, "arrival_s": 0.0, "n_sys": 36, "n": 3, "integrator": 1, "t_end": 120 * HDT, "seed": 0}
    ea = ics.three_body(40, seed=41)
    for s in range(0, 36, 3):  # 12 systems: outer planet at 99.95 AU moving outward (past 100 AU in ~3 steps)
        ea["pos"][3 * s + 2] = [99.95, 0.0, 0.0]
        ea["vel"][3 * s + 2] = [3.0, 0.0, 0.0]
    eb = ics.three_body(36, seed=42)
    with SV.Server(slots_per_pool=64, quantum_steps=25) as sv:
        ia, ib = sv.submit(ea, qa["t_end"], 1), sv.submit(eb, qb["t_end"], 1)
        sv.step()  # admits A (40) and 24 of B; the ejected systems stop and retire
        st = sv.stats()
        assert st["occupied_slots"] == 64 - 12 and st["queued"] == 1
        sv.step()  # B's last 12 systems take the freed slots; A is still running
        st = sv.stats()
        assert st["occupied_slots"] == 64 and st["queued"] == 0
        assert sv.poll(ia)[0] == SV.REQ_RUNNING
        out = {"done": {}}
        for _ in range(100):
            sv.step()
            if sv.stats()["completed"] == 2:
                break
        for r, (rid, q) in enumerate(((ia, qa), (ib, qb))):
            state, res = sv.poll(rid, q["n_sys"], q["n"])
            assert state == SV.REQ_DONE
            out["done"][r] = res
    assert np.sum(out["done"][0]["status"] == 3) == 12
    check_same([qa, qb], [ea, eb], out)


def test_stopped_systems_retire_with_their_request():
    from paper_1208_1157_gb300 import server as SV

    q = {"id": 0, "arrival_s": 0.0, "n_sys": 10, "n": 3, "integrator": 1, "t_end": 4000 * HDT, "seed": 4000}
    e = ics.three_body(10, seed=4)
    e["pos"][3 * 6 + 2] = [98.0, 0.0, 0.0]
    e["vel"][3 * 6 + 2] = [2.0, 0.0, 0.0]
    with SV.Server(slots_per_pool=64, quantum_steps=500) as sv:
        out = SV.replay(sv, [q], [e], collect=True)
    res = out["done"][0]
    assert res["status"][6] == 3 and np.all(np.delete(res["status"], 6) == 1)
    check_same([q], [e], out)


def test_cancel_and_impossible_admission():
    # fault injection on the host: a request too large for any pool is refused, a queued
    # request and a running one are cancelled; the others still finish with the same results
    from paper_1208_1157_gb300 import server as SV
    from paper_1208_1157_gb300 import swarm as S

    trace = [{"id": r, "arrival_s": 0.0, "n_sys": 40, "n": 4, "integrator": 1, "t_end": (60 + 20 * r) * HDT,
              "seed": 5000 + r} for r in range(4)]
    ens_list = [ics.request_ensemble(q) for q in trace]
    with SV.Server(slots_per_pool=96, quantum_steps=20) as sv:
        big = ics.request_ensemble({"n_sys": 97, "n": 4, "seed": 9})
        with pytest.raises(S.SwarmError):
            sv.submit(big, 1.0, 1)  # larger than a pool: never admissible
        ids = [sv.submit(e, q["t_end"], 1) for e, q in zip(ens_list, trace)]
        sv.step()  # requests 0 and 1 fit (80 of 96 slots); 2 and 3 wait
        assert sv.poll(ids[0])[0] == SV.REQ_RUNNING and sv.poll(ids[3])[0] == SV.REQ_QUEUED
        sv.cancel(ids[1])   # running: its 40 slots are freed
        sv.cancel(ids[3])   # queued: leaves the queue
        with pytest.raises(S.SwarmError):
            sv.cancel(ids[3])
        for _ in range(100):
            sv.step()
            if sv.stats()["completed"] == 2:
                break
        st = sv.stats()
        assert st["completed"] == 2 and st["cancelled"] == 2 and st["queued"] == 0
        out = {"done": {}}
        for r in (0, 2):
            state, res = sv.poll(ids[r], trace[r]["n_sys"], trace[r]["n"])
            assert state == SV.REQ_DONE
            out["done"][r] = res
        assert sv.poll(ids[1])[0] == SV.REQ_CANCELLED
        sv.release(ids[1])
    check_same([trace[0], trace[2]], [ens_list[0], ens_list[2]], {"done": {0: out["done"][0], 1: out["done"][2]}})
