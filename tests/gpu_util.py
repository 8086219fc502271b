"""Helpers shared by the GPU parity tests: run the library and the oracle on the same
seeded inputs and compare them per system."""
import math

import numpy as np

import oracle as O
from paper_1208_1157_gb300 import ics

TWO_PI = 2 * math.pi
# parity bar: positions and velocities within 1e-10 relative after 1000 steps
# (relative to the largest position / velocity of the system)
TOL = 1e-10
# A system whose own oracle result moves by more than TOL/100 when its inputs are
# perturbed by one unit in the last place is ill-conditioned (near-encounter, chaotic):
# there no implementation with another rounding order can meet TOL, and the GPU must
# instead agree to within COND_FACTOR times that measured round-off sensitivity.
COND_FACTOR = 30.0
U = 2.0 ** -53  # unit round-off


def run_gpu(ens, t_end, integrator, dt, mapping=0, ce=0.0, ej=0.0, n_corr=2, log_interval=0, log_cap=0,
            time=None, status=None, single_launch=1, rk_eps=1e-12, steps_per_launch=0):
    from paper_1208_1157_gb300 import swarm as S

    with S.Ensemble(ens) as e:
        e.set_option(S.OPT_MAPPING, mapping)
        e.set_option(S.OPT_N_CORR, n_corr)
        e.set_option(S.OPT_SINGLE_LAUNCH, single_launch)
        e.set_option(S.OPT_STEPS_PER_LAUNCH, steps_per_launch)
        e.set_tolerance(rk_eps)
        if log_cap:
            e.set_option(S.OPT_LOG_CAPACITY, log_cap)
            e.set_option(S.OPT_LOG_INTERVAL, log_interval)
        e.set_stop(ce, ej)
        if time is not None or status is not None:
            e.set_state(time=time, status=status)
        e.integrate(t_end, integrator, dt)
        out = e.state()
        out["stats"] = e.stats()
        out["energy"], out["angmom"] = e.diagnostics()
        if log_cap:
            out["logs"] = [e.log(s) for s in range(e.n_sys)]
    return out


def run_oracle(ens, t_end, integrator, dt, ce=0.0, ej=0.0, n_corr=2, log_interval=0, log_cap=0, time=None,
               status=None, rk_eps=1e-12):
    return O.integrate(ens, t_end, dt, integrator, n_corr=n_corr, ce_factor=ce, eject_radius=ej,
                       log_interval=log_interval, log_cap=log_cap, time=time, status=status, rk_eps=rk_eps)


def per_system_errors(ens, a, b):
    """max |a - b| / max |b| per system, for positions and velocities."""
    offs = np.concatenate([[0], np.cumsum(ens["n_body"])])
    ex, ev = [], []
    for s in range(len(ens["n_body"])):
        sl = slice(offs[s], offs[s + 1])
        xb, vb = b["pos"][sl], b["vel"][sl]
        ex.append(np.max(np.abs(a["pos"][sl] - xb)) / np.max(np.abs(xb)))
        ev.append(np.max(np.abs(a["vel"][sl] - vb)) / np.max(np.abs(vb)))
    return np.array(ex), np.array(ev)


def energies(ens, pos, vel):
    offs = np.concatenate([[0], np.cumsum(ens["n_body"])])
    E = np.empty(len(ens["n_body"]))
    for s in range(len(E)):
        sl = slice(offs[s], offs[s + 1])
        E[s], _ = O.energy(ens["mass"][sl], pos[sl], vel[sl])
    return E


def oracle_sensitivity(ens, t_end, integrator, dt, **kw):
    """Per-system change of the oracle's own result when every input is perturbed by
    one unit in the last place (positions up, velocities down)."""
    p = dict(ens)
    p["pos"] = ens["pos"] * (1 + 2.0 ** -52)
    p["vel"] = ens["vel"] * (1 - 2.0 ** -52)
    a = run_oracle(ens, t_end, integrator, dt, **kw)
    b = run_oracle(p, t_end, integrator, dt, **kw)
    ex, ev = per_system_errors(ens, b, a)
    return np.maximum(ex, ev)


def assert_parity(ens, g, o, tol=TOL, check_energy=True, sens=None, steps=1000, stop_time_rtol=None, max_relaxed=0.1):
    """Statuses and times equal; positions/velocities within tol (or, for systems whose
    measured round-off sensitivity `sens` exceeds tol/100, within COND_FACTOR * sens);
    the GPU's relative energy error within 2x the oracle's, or below the round-off bound
    steps * u when the oracle's own error is at that level.

    max_relaxed caps the relaxation where the contract is strict: of the systems that ran
    the whole call without a stop (the non-close-encounter systems), at most this fraction
    may exceed tol at all (within the sensitivity bound above); the counts are printed and
    reported in the failure message.  Systems that stopped on the way are not capped.

    stop_time_rtol: for an integrator whose step sizes come from an error estimate (the
    adaptive Runge-Kutta step), the estimate is a short sum of large terms that cancel, so
    its rounding fixes each step size only to ~1e-9 relative: a system that stops on the
    way then stops at a time that may differ by that much.  Such systems get this time
    tolerance, and their states the distance covered in the time difference."""
    assert np.array_equal(g["status"], o["status"]), (
        f"status mismatch at systems {np.nonzero(g['status'] != o['status'])[0][:10]}: "
        f"gpu {g['status'][g['status'] != o['status']][:10]} oracle {o['status'][g['status'] != o['status']][:10]}")
    ex, ev = per_system_errors(ens, g, o)
    bound = np.full(len(ex), tol)
    tbound = np.full(len(ex), 1e-13)
    if sens is not None:
        ill = sens > tol / 100
        bound = np.where(ill, np.maximum(tol, COND_FACTOR * sens), tol)
        # an adaptive integrator's stop time follows the trajectory: same bound there
        tbound = np.where(ill, np.maximum(1e-13, COND_FACTOR * sens), 1e-13)
    dt_rel = np.abs(g["time"] - o["time"]) / np.maximum(np.abs(o["time"]), 1.0)
    if stop_time_rtol is not None:
        stopped = o["status"] >= 2
        tbound = np.where(stopped, np.maximum(tbound, stop_time_rtol), tbound)
        # distance covered in the time difference, relative to the system's size
        offs = np.concatenate([[0], np.cumsum(ens["n_body"])])
        rate = np.array([np.abs(o["vel"][offs[k]:offs[k + 1]]).max() / np.abs(o["pos"][offs[k]:offs[k + 1]]).max()
                         for k in range(len(offs) - 1)])  # ~ orbital frequency: |dx|/|x|, |dv|/|v| per unit time
        bound = np.where(stopped, bound + 10.0 * np.abs(g["time"] - o["time"]) * rate, bound)
    assert np.all(dt_rel <= tbound), f"time mismatch at {np.nonzero(dt_rel > tbound)[0][:10]}: {dt_rel[dt_rel > tbound][:5]}"
    err = np.maximum(ex, ev)
    if sens is not None:
        ran = o["status"] <= 1  # reached the end time: no stop on the way
        over = err > tol
        n_ran, n_over = int(ran.sum()), int((over & ran).sum())
        msg = (f"strict {tol:g} bar met by {n_ran - n_over} of {n_ran} systems that ran the whole call "
               f"({n_over} within {COND_FACTOR:g}x the oracle's own 1-ulp sensitivity, cap {max_relaxed:.0%}); "
               f"{int((over & ~ran).sum())} of {int((~ran).sum())} stopped systems above {tol:g}")
        print("parity:", msg)
        assert n_over <= max_relaxed * n_ran, msg
    r = err / bound
    worst = int(np.argmax(r))
    sw = "n/a" if sens is None else f"{sens[worst]:.3e}"
    assert r.max() <= 1.0, f"worst system {worst}: pos {ex[worst]:.3e} vel {ev[worst]:.3e} bound {bound[worst]:.3e} (sensitivity {sw})"
    if check_energy:
        E0 = energies(ens, ens["pos"], ens["vel"])
        Eg = energies(ens, g["pos"], g["vel"])
        Eo = energies(ens, o["pos"], o["vel"])
        dg = np.abs(Eg / E0 - 1)
        do = np.abs(Eo / E0 - 1)
        bad = dg > np.maximum(2 * do, steps * U)
        assert not bad.any(), f"energy error above 2x the oracle's at {np.nonzero(bad)[0][:10]}: {dg[bad][:5]} vs {do[bad][:5]}"
    return ex, ev


def block_ring_wave(n, sms):
    """Systems in one wave of the CTA-packed body-per-lane kernels (hermite_block.cuh,
    rkck_block.cuh): 256-thread CTAs, one per SM, where they pack more lanes than 128,
    else two CTAs of 128 per SM; floor(T / n) systems per CTA.  Bins of at least this
    many systems of n bodies take those kernels when the warp ring (floor(32/n) systems
    per warp, 8 warps per SM) needs more waves or as many with 10 % fewer lanes busy
    (n = 7, 9, 11..15 here)."""
    T = 256 if (256 // n) * n > 2 * ((128 // n) * n) else 128
    return (256 // T) * sms * (T // n)
