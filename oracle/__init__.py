"""CPU oracle for the Swarm-NG integrators — TEST INFRASTRUCTURE ONLY.

A plain single-threaded FP64 C restatement of the paper's method (oracle.c); this
module compiles it with gcc (no FMA contraction, so results are the same on x86 and
Arm) and wraps it with ctypes.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package; the library never does.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
HDR = os.path.join(HERE, "oracle.h")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")

ACTIVE, DONE, CLOSE_ENCOUNTER, EJECTED, KEPLER_NOCONV, NONFINITE = range(6)
HERMITE, MVS_DH, MVS_JACOBI, HERMITE_ADAPTIVE, RKCK, RKCK_ADAPTIVE = 1, 2, 3, 4, 5, 6
CORR_KOKUBO, CORR_PRINTED = 0, 1

_lock = threading.Lock()
_lib = None


# the oracle's build: strict IEEE order (no contraction into FMAs, no fast math), the same
# results on x86 and Arm; also what the CPU baseline times
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC"]


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so if missing or stale."""
    os.makedirs(OUT_DIR, exist_ok=True)
    stale = force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(SRC), os.path.getmtime(HDR))
    if stale:
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["gcc"] + CFLAGS + ["-shared", "-o", tmp, SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    return LIB


def lib():
    """The compiled oracle; ORACLE_LIB names another build of it (the mutation tests)."""
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(os.environ.get("ORACLE_LIB") or build())
            _declare(_lib)
    return _lib


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def _declare(L):
    L.or_accjerk.argtypes = [C.c_int, _dp, _dp, _dp, _dp, _dp]
    L.or_acc.argtypes = [C.c_int, _dp, _dp, _dp]
    L.or_hermite_step.argtypes = [C.c_int, _dp, _dp, _dp, _dp, _dp, C.c_double, C.c_int, C.c_int]
    L.or_energy.argtypes = [C.c_int, _dp, _dp, _dp, _dp, _dp]
    L.or_adaptive_dt.argtypes = [C.c_int, _dp, _dp, C.c_double]
    L.or_adaptive_dt.restype = C.c_double
    L.or_monitor.argtypes = [C.c_int, _dp, _dp, _dp, C.c_double, C.c_double]
    L.or_monitor.restype = C.c_int
    L.or_stumpff.argtypes = [C.c_double, _dp, _dp]
    L.or_kepler_drift.argtypes = [C.c_double, _dp, _dp, C.c_double, _ip]
    L.or_kepler_drift.restype = C.c_int
    for f in ("or_inertial_to_dh", "or_dh_to_inertial", "or_inertial_to_jacobi", "or_jacobi_to_inertial"):
        getattr(L, f).argtypes = [C.c_int, _dp, _dp, _dp, _dp, _dp]
    L.or_mvs_dh_step.argtypes = [C.c_int, _dp, _dp, _dp, _dp, C.c_double]
    L.or_mvs_dh_step.restype = C.c_int
    L.or_mvs_jacobi_step.argtypes = [C.c_int, _dp, _dp, _dp, _dp, C.c_double]
    L.or_mvs_jacobi_step.restype = C.c_int
    L.or_dh_interaction_acc.argtypes = [C.c_int, _dp, _dp, _dp]
    L.or_jacobi_interaction_acc.argtypes = [C.c_int, _dp, _dp, _dp]
    L.or_integrate_ensemble.argtypes = [C.c_int, _ip, _dp, _dp, _dp, _dp, _ip, C.c_double, C.c_double, C.c_int,
                                        C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int, _dp, _ip,
                                        C.POINTER(C.c_longlong), C.c_double]
    L.or_integrate_ensemble.restype = C.c_int
    L.or_observe_rv_ensemble.argtypes = [C.c_int, _ip, _dp, _dp, _dp, _dp, _ip, _dp, C.c_int, C.c_double, C.c_int,
                                         C.c_double, C.c_double, C.c_double, _dp, _dp]
    L.or_observe_rv_ensemble.restype = C.c_int
    L.or_rkck_tableau.argtypes = [_dp, _dp, _dp, _dp]
    L.or_rkck_step.argtypes = [C.c_int, _dp, _dp, _dp, C.c_double, _dp]
    L.or_rkck_step.restype = C.c_double


def _d(a):
    return a.ctypes.data_as(_dp)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64).copy()
    return a if shape is None else a.reshape(shape)


# ---------------------------------------------------------------- single system
def accjerk(m, x, v):
    m, x, v = _f64(m), _f64(x, (-1, 3)), _f64(v, (-1, 3))
    a, j = np.zeros_like(x), np.zeros_like(x)
    lib().or_accjerk(len(m), _d(m), _d(x), _d(v), _d(a), _d(j))
    return a, j


def acc(m, x):
    m, x = _f64(m), _f64(x, (-1, 3))
    a = np.zeros_like(x)
    lib().or_acc(len(m), _d(m), _d(x), _d(a))
    return a


def hermite_step(m, x, v, a0, j0, dt, n_corr=2, form=CORR_KOKUBO):
    m, x, v, a0, j0 = _f64(m), _f64(x, (-1, 3)), _f64(v, (-1, 3)), _f64(a0, (-1, 3)), _f64(j0, (-1, 3))
    lib().or_hermite_step(len(m), _d(m), _d(x), _d(v), _d(a0), _d(j0), float(dt), int(n_corr), int(form))
    return x, v, a0, j0


def adaptive_dt(a0, j0, tau):
    a0, j0 = _f64(a0, (-1, 3)), _f64(j0, (-1, 3))
    return float(lib().or_adaptive_dt(len(a0), _d(a0), _d(j0), float(tau)))


def energy(m, x, v):
    m, x, v = _f64(m), _f64(x, (-1, 3)), _f64(v, (-1, 3))
    E = np.zeros(1)
    L = np.zeros(3)
    lib().or_energy(len(m), _d(m), _d(x), _d(v), _d(E), _d(L))
    return float(E[0]), L


def monitor(m, x, v, ce_factor=0.0, eject_radius=0.0):
    m, x, v = _f64(m), _f64(x, (-1, 3)), _f64(v, (-1, 3))
    return int(lib().or_monitor(len(m), _d(m), _d(x), _d(v), float(ce_factor), float(eject_radius)))


def stumpff(z):
    c2, c3 = C.c_double(), C.c_double()
    lib().or_stumpff(float(z), C.byref(c2), C.byref(c3))
    return c2.value, c3.value


def kepler_drift(mu, r, v, dt):
    r, v = _f64(r), _f64(v)
    it = C.c_int()
    st = lib().or_kepler_drift(float(mu), _d(r), _d(v), float(dt), C.byref(it))
    return r, v, int(st), it.value


def _conv(name, m, a, b):
    m, a, b = _f64(m), _f64(a, (-1, 3)), _f64(b, (-1, 3))
    p, q = np.zeros_like(a), np.zeros_like(b)
    getattr(lib(), name)(len(m), _d(m), _d(a), _d(b), _d(p), _d(q))
    return p, q


def inertial_to_dh(m, x, v):
    return _conv("or_inertial_to_dh", m, x, v)


def dh_to_inertial(m, q, u):
    return _conv("or_dh_to_inertial", m, q, u)


def inertial_to_jacobi(m, x, v):
    return _conv("or_inertial_to_jacobi", m, x, v)


def jacobi_to_inertial(m, r, w):
    return _conv("or_jacobi_to_inertial", m, r, w)


def dh_interaction_acc(m, q):
    m, q = _f64(m), _f64(q, (-1, 3))
    a = np.zeros_like(q)
    lib().or_dh_interaction_acc(len(m), _d(m), _d(q), _d(a))
    return a


def jacobi_interaction_acc(m, r):
    m, r = _f64(m), _f64(r, (-1, 3))
    a = np.zeros_like(r)
    lib().or_jacobi_interaction_acc(len(m), _d(m), _d(r), _d(a))
    return a


def mvs_step(kind, m, q, u, acc_cache, dt):
    """One MVS step on coordinates (q, u) with the acceleration cache; returns new arrays."""
    m, q, u, a = _f64(m), _f64(q, (-1, 3)), _f64(u, (-1, 3)), _f64(acc_cache, (-1, 3))
    f = lib().or_mvs_dh_step if kind == MVS_DH else lib().or_mvs_jacobi_step
    st = f(len(m), _d(m), _d(q), _d(u), _d(a), float(dt))
    return q, u, a, int(st)


def rkck_tableau():
    c, a, b5, b4 = np.zeros(6), np.zeros(36), np.zeros(6), np.zeros(6)
    lib().or_rkck_tableau(_d(c), _d(a), _d(b5), _d(b4))
    return c, a.reshape(6, 6), b5, b4


def rkck_step(m, x, v, h):
    """One Cash-Karp step; returns (x, v, scaled error, error vector [2n][3])."""
    m, x, v = _f64(m), _f64(x, (-1, 3)), _f64(v, (-1, 3))
    err = np.zeros((2 * len(m), 3))
    e = lib().or_rkck_step(len(m), _d(m), _d(x), _d(v), float(h), _d(err))
    return x, v, float(e), err


# ---------------------------------------------------------------- ensembles
def integrate(ens: dict, t_end: float, dt: float, integrator: int = HERMITE, n_corr: int = 2,
              corr_form: int = CORR_KOKUBO, ce_factor: float = 0.0, eject_radius: float = 0.0,
              log_interval: int = 0, log_cap: int = 0, time=None, status=None, rk_eps: float = 1e-12) -> dict:
    """Integrate every system of `ens` (the ics layout) from `time` (default 0) to t_end."""
    n_body = np.ascontiguousarray(ens["n_body"], dtype=np.int32)
    S = len(n_body)
    mass = _f64(ens["mass"])
    pos = _f64(ens["pos"], (-1, 3))
    vel = _f64(ens["vel"], (-1, 3))
    tm = np.zeros(S) if time is None else _f64(time)
    stt = np.zeros(S, dtype=np.int32) if status is None else np.ascontiguousarray(status, dtype=np.int32).copy()
    cap = max(int(log_cap), 0) if log_interval > 0 else 0
    log = np.zeros((S, max(cap, 1), 5))
    cnt = np.zeros(S, dtype=np.int32)
    kit = C.c_longlong(0)
    rc = lib().or_integrate_ensemble(S, n_body.ctypes.data_as(_ip), _d(mass), _d(pos), _d(vel), _d(tm),
                                     stt.ctypes.data_as(_ip), float(t_end), float(dt), int(integrator),
                                     int(n_corr), int(corr_form), float(ce_factor), float(eject_radius),
                                     int(log_interval), max(cap, 1), _d(log), cnt.ctypes.data_as(_ip),
                                     C.byref(kit), float(rk_eps))
    if rc != 0:
        raise ValueError(f"oracle integrate rejected its arguments (rc={rc})")
    return {"pos": pos, "vel": vel, "time": tm, "status": stt, "log": log[:, :cap], "log_count": cnt,
            "kepler_iters": kit.value}


def observe_rv(ens: dict, t_obs, dt: float, integrator: int = HERMITE, los=(0.0, 0.0, 1.0), ce_factor: float = 0.0,
               eject_radius: float = 0.0, rk_eps: float = 1e-12) -> dict:
    """Radial velocity of every system's central body at each observation time:
    rv [n_obs][n_sys], plus the final state."""
    n_body = np.ascontiguousarray(ens["n_body"], dtype=np.int32)
    S = len(n_body)
    mass = _f64(ens["mass"])
    pos = _f64(ens["pos"], (-1, 3))
    vel = _f64(ens["vel"], (-1, 3))
    tm = np.zeros(S)
    stt = np.zeros(S, dtype=np.int32)
    t_obs = _f64(t_obs)
    los = _f64(los)
    rv = np.zeros((len(t_obs), S))
    rc = lib().or_observe_rv_ensemble(S, n_body.ctypes.data_as(_ip), _d(mass), _d(pos), _d(vel), _d(tm),
                                      stt.ctypes.data_as(_ip), _d(t_obs), len(t_obs), float(dt), int(integrator),
                                      float(ce_factor), float(eject_radius), float(rk_eps), _d(los), _d(rv))
    if rc != 0:
        raise ValueError(f"oracle observe_rv rejected its arguments (rc={rc})")
    return {"rv": rv, "pos": pos, "vel": vel, "time": tm, "status": stt}
