"""Seeded synthetic initial conditions for few-body planetary ensembles.

This module produces inputs only: masses, positions and velocities of many
independent planetary systems, drawn from a counter-based SplitMix64 stream so
that every value is a pure function of (seed, system index, draw index).  It holds
none of the integration arithmetic; both the CUDA path and the CPU oracle take
its arrays as given.

Units follow Sec. 2.1 of the paper (Eq. 1 with G = 1): lengths in AU, masses in
solar masses, one year = 2*pi time units.  Body 0 of every system is the star.

Ensemble layout returned by every generator (a dict):
  n_body  int32  [S]       bodies per system (2..32)
  mass    float64[B]       B = sum(n_body), systems back to back, star first
  pos     float64[B, 3]    barycentric positions
  vel     float64[B, 3]    barycentric velocities

Recipe (the paper's own ICs of Sec. 5.1 plus the workload families used for
measurement; every choice beyond the paper is named here):
  * planets get osculating astrocentric elements (a, e, i, Omega, omega, E) with
    mu = m0 + m_i, converted with the two-body closed form; the phase is drawn as
    the eccentric anomaly E ~ U[0, 2 pi) so that no Kepler equation is solved here;
  * the whole system is then shifted to the barycentric frame (zero total
    momentum), so energy and angular momentum tests are frame-clean.
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


# ---------------------------------------------------------------------------
# counter-based SplitMix64 (Steele, Lea & Flood 2014, "Fast splittable
# pseudorandom number generators"): output = mix(key + (k + 1) * golden)
# ---------------------------------------------------------------------------
def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _keys(seed: int, idx: np.ndarray) -> np.ndarray:
    """One 64-bit key per stream index (system), derived from the seed."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        base = _mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _GOLDEN + np.uint64(0x632BE59BD9B4E019))
        return _mix64(base ^ _mix64((idx + np.uint64(1)) * _GOLDEN))


def uniform(seed: int, idx: np.ndarray, k: int) -> np.ndarray:
    """k-th U[0,1) draw of each stream in `idx` (53-bit mantissa)."""
    key = _keys(seed, idx)
    with np.errstate(over="ignore"):
        z = _mix64(key + np.uint64(k + 1) * _GOLDEN)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# ---------------------------------------------------------------------------
# two-body elements -> Cartesian (closed form in the eccentric anomaly)
# ---------------------------------------------------------------------------
def elements_to_cartesian(mu, a, e, inc, node, peri, ecc_anom):
    """Astrocentric position/velocity of a bound orbit from (a, e, i, Omega, omega, E).

    Standard two-body relations (e.g. Murray & Dermott 2000, Sec. 2.5): in-plane
    position a(cos E - e), a sqrt(1-e^2) sin E; rotation R_z(Omega) R_x(i) R_z(omega).
    """
    mu, a, e, inc, node, peri, E = np.broadcast_arrays(*(np.asarray(t, dtype=np.float64) for t in (mu, a, e, inc, node, peri, ecc_anom)))
    cE, sE = np.cos(E), np.sin(E)
    b = a * np.sqrt(1.0 - e * e)
    xo = a * (cE - e)
    yo = b * sE
    edot = np.sqrt(mu / (a * a * a)) / (1.0 - e * cE)
    vxo = -a * sE * edot
    vyo = b * cE * edot
    cO, sO = np.cos(node), np.sin(node)
    cw, sw = np.cos(peri), np.sin(peri)
    ci, si = np.cos(inc), np.sin(inc)
    # columns of R_z(Omega) R_x(i) R_z(omega) acting on the in-plane x and y axes
    px = np.stack([cO * cw - sO * sw * ci, sO * cw + cO * sw * ci, sw * si], axis=-1)
    py = np.stack([-cO * sw - sO * cw * ci, -sO * sw + cO * cw * ci, cw * si], axis=-1)
    pos = xo[..., None] * px + yo[..., None] * py
    vel = vxo[..., None] * px + vyo[..., None] * py
    return pos, vel


def _to_barycentric(n_body, mass, pos, vel):
    offs = np.concatenate([[0], np.cumsum(n_body)])
    sys_of_body = np.repeat(np.arange(len(n_body)), n_body)
    mtot = np.add.reduceat(mass, offs[:-1])
    mx = np.zeros((len(n_body), 3))
    mv = np.zeros((len(n_body), 3))
    np.add.at(mx, sys_of_body, mass[:, None] * pos)
    np.add.at(mv, sys_of_body, mass[:, None] * vel)
    pos = pos - (mx / mtot[:, None])[sys_of_body]
    vel = vel - (mv / mtot[:, None])[sys_of_body]
    return pos, vel


def _assemble(n_body, m0, mp, a, e, inc, node, peri, E):
    """n_body [S]; planet arrays are [S, max_n-1] with valid entries j < n_body-1."""
    S = len(n_body)
    B = int(np.sum(n_body))
    mass = np.empty(B)
    pos = np.zeros((B, 3))
    vel = np.zeros((B, 3))
    offs = np.concatenate([[0], np.cumsum(n_body)]).astype(np.int64)
    mass[offs[:-1]] = m0
    npl = n_body - 1
    for j in range(int(npl.max())):
        sel = np.nonzero(npl > j)[0]
        if len(sel) == 0:
            continue
        rows = offs[sel] + 1 + j
        mu = m0 + mp[sel, j]
        p, v = elements_to_cartesian(mu, a[sel, j], e[sel, j], inc[sel, j], node[sel, j], peri[sel, j], E[sel, j])
        mass[rows] = mp[sel, j]
        pos[rows] = p
        vel[rows] = v
    pos, vel = _to_barycentric(n_body, mass, pos, vel)
    return {"n_body": n_body.astype(np.int32), "mass": mass, "pos": pos, "vel": vel}


def _angles(seed, idx, base_k, shape_j):
    """inclination U(0, 0.01) rad, Omega/omega/E ~ U[0, 2 pi) for planets 0..shape_j-1."""
    inc = np.stack([0.01 * uniform(seed, idx, base_k + 4 * j + 0) for j in range(shape_j)], axis=1)
    node = np.stack([TWO_PI * uniform(seed, idx, base_k + 4 * j + 1) for j in range(shape_j)], axis=1)
    peri = np.stack([TWO_PI * uniform(seed, idx, base_k + 4 * j + 2) for j in range(shape_j)], axis=1)
    E = np.stack([TWO_PI * uniform(seed, idx, base_k + 4 * j + 3) for j in range(shape_j)], axis=1)
    return inc, node, peri, E


def _log_uniform(u, lo, hi):
    return np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))


# ---------------------------------------------------------------------------
# workload families
# ---------------------------------------------------------------------------
def three_body(n_sys: int, seed: int) -> dict:
    """Star (1 Msun) + 2 planets: masses log-U(1e-5, 1e-3), a1 = 1, a2 ~ U(1.6, 3),
    e ~ U(0, 0.05), i ~ U(0, 0.01) rad, Omega/omega/E ~ U[0, 2 pi).
    1024 systems with seed 1 is the small parity case, 131072 with seed 2 the
    paper-shaped ensemble of Table 3 / Table 4."""
    idx = np.arange(n_sys)
    n_body = np.full(n_sys, 3, dtype=np.int32)
    mp = np.stack([_log_uniform(uniform(seed, idx, j), 1e-5, 1e-3) for j in range(2)], axis=1)
    a = np.stack([np.ones(n_sys), 1.6 + 1.4 * uniform(seed, idx, 2)], axis=1)
    e = np.stack([0.05 * uniform(seed, idx, 3 + j) for j in range(2)], axis=1)
    inc, node, peri, E = _angles(seed, idx, 8, 2)
    return _assemble(n_body, 1.0, mp, a, e, inc, node, peri, E)


def _hill_spaced(n_body, seed, idx, e_max, base_k, m_lo=1e-5, m_hi=1e-3, stride=20, k_lo=3.0, k_hi=8.0):
    """a_1 = 1; a_{j+1} = a_j (1 + K h/2)/(1 - K h/2), h = ((m_j + m_{j+1})/3)^(1/3), K ~ U(k_lo, k_hi);
    masses log-U(m_lo, m_hi).  Draw k of planet j: mass base_k + j, e base_k + stride + j,
    K base_k + 2 stride + j, angles from base_k + 3 stride (stride > planets per system)."""
    S = len(n_body)
    P = int(n_body.max()) - 1
    assert P < stride
    mp = np.zeros((S, P))
    a = np.zeros((S, P))
    e = np.zeros((S, P))
    for j in range(P):
        mp[:, j] = _log_uniform(uniform(seed, idx, base_k + j), m_lo, m_hi)
        e[:, j] = e_max * uniform(seed, idx, base_k + stride + j)
    a[:, 0] = 1.0
    for j in range(1, P):
        K = k_lo + (k_hi - k_lo) * uniform(seed, idx, base_k + 2 * stride + j)
        h = np.cbrt((mp[:, j - 1] + mp[:, j]) / 3.0)
        a[:, j] = a[:, j - 1] * (1.0 + 0.5 * K * h) / (1.0 - 0.5 * K * h)
    inc, node, peri, E = _angles(seed, idx, base_k + 3 * stride, P)
    return mp, a, e, inc, node, peri, E


def ragged(n_sys: int, seed: int, n_min: int = 3, n_max: int = 15) -> dict:
    """n ~ U{n_min..n_max} bodies (1 star + n-1 planets), masses log-U(1e-5, 1e-3),
    Hill-spaced semi-major axes (K ~ U(3, 8) mutual Hill radii), e ~ U(0, 0.1)."""
    idx = np.arange(n_sys)
    n_body = (n_min + np.floor((n_max - n_min + 1) * uniform(seed, idx, 0))).astype(np.int32)
    mp, a, e, inc, node, peri, E = _hill_spaced(n_body, seed, idx, 0.1, 1)
    return _assemble(n_body, 1.0, mp, a, e, inc, node, peri, E)


def ragged_wide(n_sys: int, seed: int, n_min: int = 16, n_max: int = 32) -> dict:
    """Larger systems: n ~ U{n_min..n_max} (up to 31 planets), masses log-U(1e-7, 1e-5)
    (Mars to Neptune mass in solar units), Hill spacing as in `ragged` (K ~ U(3, 8)),
    e ~ U(0, 0.1); the outermost orbit stays within ~15 AU."""
    idx = np.arange(n_sys)
    n_body = (n_min + np.floor((n_max - n_min + 1) * uniform(seed, idx, 0))).astype(np.int32)
    mp, a, e, inc, node, peri, E = _hill_spaced(n_body, seed, idx, 0.1, 1, m_lo=1e-7, m_hi=1e-5, stride=40)
    return _assemble(n_body, 1.0, mp, a, e, inc, node, peri, E)


def mvs_compact(n_sys: int, seed: int, n: int = 8, a_lim: float = 50.0, k_lo: float = 3.0, k_hi: float = 8.0,
                m_lo: float = 1e-5, m_hi: float = 1e-3) -> dict:
    """n bodies, Hill spacing as in `ragged` (K ~ U(k_lo, k_hi) mutual Hill radii, planet
    masses log-U(m_lo, m_hi)), e ~ U(0, 0.1);
    a system whose outermost apocentre a (1 + e) reaches `a_lim` AU is redrawn from the
    next attempt of its own stream."""
    S = n_sys
    n_body = np.full(S, n, dtype=np.int32)
    out = None
    todo = np.arange(S)
    attempt = 0
    while len(todo):
        nb = n_body[todo]
        # attempt r of system s uses stream index s + r * 2^32
        idx = todo.astype(np.uint64) + np.uint64(attempt) * np.uint64(1 << 32)
        parts = _hill_spaced(nb, seed, idx, 0.1, 1, m_lo=m_lo, m_hi=m_hi, k_lo=k_lo, k_hi=k_hi)
        if out is None:
            out = [np.zeros((S,) + p.shape[1:]) for p in parts]
        apo = parts[1][:, -1] * (1.0 + parts[2][:, -1])
        ok = apo < a_lim
        for o, p in zip(out, parts):
            o[todo[ok]] = p[ok]
        todo = todo[~ok]
        attempt += 1
        if attempt > 1000:
            raise RuntimeError("mvs_compact: could not draw compact systems")
    return _assemble(n_body, 1.0, *out)


def paper_standard(n_sys: int, n: int = 3, planet_mass: float = 1e-3, spacing: float = 0.4) -> dict:
    """The paper's verification ICs (Sec. 5.1): m0 = 1, equal planet masses, circular
    coplanar orbits at a_i = (1 + alpha)^(i-1).  The circular speed is taken in G = 1
    units, sqrt(m0 / a_i) (the paper's printed 2 pi (m0/a^3)^(1/2) mixes year units);
    the star is then moved so that the system is barycentric.  Planet i starts at
    phase angle 0 (all planets aligned), identical for every system."""
    n_body = np.full(n_sys, n, dtype=np.int32)
    P = n - 1
    mp = np.full((n_sys, P), planet_mass)
    a = np.tile((1.0 + spacing) ** np.arange(P), (n_sys, 1))
    z = np.zeros((n_sys, P))
    # circular orbit about the star alone (mu = m0): speed sqrt(m0 / a)
    pos = np.zeros((n_sys * n, 3))
    vel = np.zeros((n_sys * n, 3))
    mass = np.empty(n_sys * n)
    for s in range(n_sys):
        o = s * n
        mass[o] = 1.0
        for j in range(P):
            mass[o + 1 + j] = planet_mass
            pos[o + 1 + j, 0] = a[s, j]
            vel[o + 1 + j, 1] = math.sqrt(1.0 / a[s, j])
    pos, vel = _to_barycentric(n_body, mass, pos, vel)
    del z
    return {"n_body": n_body, "mass": mass, "pos": pos, "vel": vel}


def two_body(a: float, e: float, m0: float = 1.0, m1: float = 1e-3, E0: float = 0.0) -> dict:
    """One star + one planet on an (a, e) orbit starting at eccentric anomaly E0, barycentric."""
    n_body = np.array([2], dtype=np.int32)
    p, v = elements_to_cartesian(m0 + m1, a, e, 0.0, 0.0, 0.0, E0)
    mass = np.array([m0, m1])
    pos = np.zeros((2, 3))
    vel = np.zeros((2, 3))
    pos[1] = p
    vel[1] = v
    pos, vel = _to_barycentric(n_body, mass, pos, vel)
    return {"n_body": n_body, "mass": mass, "pos": pos, "vel": vel}


def subset(ens: dict, systems) -> dict:
    """The listed systems of an ensemble, in the listed order."""
    systems = np.asarray(systems, dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(ens["n_body"])]).astype(np.int64)
    rows = np.concatenate([np.arange(offs[s], offs[s + 1]) for s in systems]) if len(systems) else np.zeros(0, np.int64)
    return {"n_body": ens["n_body"][systems].copy(), "mass": ens["mass"][rows].copy(),
            "pos": ens["pos"][rows].copy(), "vel": ens["vel"][rows].copy()}


def concat(*ens: dict) -> dict:
    return {k: np.concatenate([e[k] for e in ens]) for k in ("n_body", "mass", "pos", "vel")}


# ---------------------------------------------------------------------------
# serving trace
# ---------------------------------------------------------------------------
def serving_trace(n_req: int = 512, seed: int = 5, rate: float = 200.0, t_scale: float = 1.0,
                  max_systems: int = 4096) -> list[dict]:
    """Poisson arrivals (mean `rate` per second); each request has a log-uniform
    size in 1..max_systems systems, one body count n ~ U{3..15}, integrator 50/50
    Hermite / MVS (democratic heliocentric), and t_end log-U(10, 1e4) inner periods
    (2 pi each) divided by `t_scale`.  Request r draws from stream index r; its
    systems are `ragged`-family systems of that single n with seed (seed, r)."""
    idx = np.arange(n_req)
    gaps = -np.log1p(-uniform(seed, idx, 0)) / rate
    arrival = np.cumsum(gaps) - gaps[0]
    size = np.clip(np.floor(np.exp(uniform(seed, idx, 1) * math.log(max_systems + 1))), 1, max_systems).astype(np.int64)
    n = (3 + np.floor(13 * uniform(seed, idx, 2))).astype(np.int32)
    integ = np.where(uniform(seed, idx, 3) < 0.5, 1, 2).astype(np.int32)
    periods = _log_uniform(uniform(seed, idx, 4), 10.0, 1e4) / t_scale
    reqs = []
    for r in range(n_req):
        reqs.append({"id": r, "arrival_s": float(arrival[r]), "n_sys": int(size[r]), "n": int(n[r]),
                     "integrator": int(integ[r]), "t_end": float(TWO_PI * periods[r]),
                     "seed": (seed << 20) + r})
    return reqs


def request_ensemble(req: dict) -> dict:
    """The systems of one serving request (all with the request's body count)."""
    S = req["n_sys"]
    idx = np.arange(S)
    n_body = np.full(S, req["n"], dtype=np.int32)
    mp, a, e, inc, node, peri, E = _hill_spaced(n_body, req["seed"], idx, 0.1, 1)
    return _assemble(n_body, 1.0, mp, a, e, inc, node, peri, E)
