"""ctypes binding of libswarm_gb300.so (include/swarm.h): argument marshalling only.

Every computation runs in the library's sm_103a kernels; this module converts numpy
arrays / torch tensors to pointers and return codes to exceptions.  If the compiled
library is missing, the first call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libswarm_gb300.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ESTATE = 0, -1, -2, -3, -4, -5
HERMITE4, MVS_DH, MVS_JACOBI, HERMITE4_ADAPTIVE, RKCK, RKCK_ADAPTIVE = 1, 2, 3, 4, 5, 6
ACTIVE, DONE, CLOSE_ENCOUNTER, EJECTED, KEPLER_NOCONV, NONFINITE, SPAN_LIMIT = range(7)
MAP_AUTO, MAP_SYSTEM_PER_LANE, MAP_BODY_PER_LANE, MAP_PLAIN_PER_STEP = range(4)
OPT_MAPPING, OPT_N_CORR, OPT_LOG_INTERVAL, OPT_LOG_CAPACITY, OPT_STEPS_PER_LAUNCH, OPT_SINGLE_LAUNCH, OPT_CTAS_PER_SM, OPT_CORRECTOR = range(1, 9)

# every symbol include/swarm.h declares (checked by the ABI test)
EXPORTS = (
    "swarm_create_ensemble", "swarm_set_stop", "swarm_set_option", "swarm_set_tolerance", "swarm_query_rv",
    "swarm_observe_rv", "swarm_integrate", "swarm_integrate_async",
    "swarm_synchronize", "swarm_set_state", "swarm_query_state", "swarm_query_state_dev", "swarm_set_state_dev", "swarm_query_diagnostics",
    "swarm_query_log", "swarm_query_stats", "swarm_ensemble_size", "swarm_destroy_ensemble", "swarm_tuner_choice",
    "swarm_tuner_load", "swarm_tuner_save", "swarm_fp64_peak", "swarm_last_error", "swarm_version",
    "swarm_hermite_integrate_noalloc",
)


class SwarmError(RuntimeError):
    def __init__(self, rc, msg):
        super().__init__(f"swarm error {rc}: {msg}")
        self.rc = rc


class Stats(C.Structure):
    _fields_ = [("system_steps", C.c_int64), ("pair_evaluations", C.c_int64), ("kepler_iterations", C.c_int64),
                ("kernel_launches", C.c_int64), ("kernel_ms", C.c_double)]


_lock = threading.Lock()
_lib = None
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_vp = C.c_void_p


def lib():
    """The loaded library; raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run paper_1208_1157_gb300.build.build() "
                                   "(nvcc, sm_103a) first; there is no CPU fallback")
            L = C.CDLL(LIB_PATH)
            L.swarm_create_ensemble.argtypes = [C.c_int32, _ip, _dp, _dp, _dp, C.c_double, _vp, C.POINTER(_vp)]
            L.swarm_set_stop.argtypes = [_vp, C.c_double, C.c_double]
            L.swarm_set_option.argtypes = [_vp, C.c_int, C.c_int64]
            L.swarm_set_tolerance.argtypes = [_vp, C.c_double]
            L.swarm_query_rv.argtypes = [_vp, _dp, _dp]
            L.swarm_observe_rv.argtypes = [_vp, _dp, C.c_int32, C.c_int, C.c_double, _dp, _dp]
            L.swarm_integrate.argtypes = [_vp, C.c_double, C.c_int, C.c_double]
            L.swarm_integrate_async.argtypes = [_vp, C.c_double, C.c_int, C.c_double]
            L.swarm_synchronize.argtypes = [_vp]
            L.swarm_set_state.argtypes = [_vp, _dp, _dp, _dp, _ip]
            L.swarm_query_state.argtypes = [_vp, _dp, _dp, _dp, _ip]
            L.swarm_query_state_dev.argtypes = [_vp, _vp, _vp, _vp, _vp]
            L.swarm_set_state_dev.argtypes = [_vp, _vp, _vp, _vp, _vp]
            L.swarm_query_diagnostics.argtypes = [_vp, _dp, _dp]
            L.swarm_query_log.argtypes = [_vp, C.c_int32, _dp, C.c_int32, _ip]
            L.swarm_query_stats.argtypes = [_vp, C.POINTER(Stats)]
            L.swarm_ensemble_size.argtypes = [_vp]
            L.swarm_ensemble_size.restype = C.c_int32
            L.swarm_destroy_ensemble.argtypes = [_vp]
            L.swarm_destroy_ensemble.restype = None
            L.swarm_tuner_choice.argtypes = [C.c_int32, C.c_int, C.c_int32, _vp, _ip, _ip]
            L.swarm_tuner_load.argtypes = [C.c_char_p]
            L.swarm_tuner_save.argtypes = [C.c_char_p]
            L.swarm_fp64_peak.argtypes = [C.c_double, _vp, _dp]
            L.swarm_last_error.restype = C.c_char_p
            L.swarm_version.restype = C.c_char_p
            _lib = L
    return _lib


def _check(rc):
    if rc != OK:
        raise SwarmError(rc, lib().swarm_last_error().decode())


def _d(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


class Ensemble:
    """A device-resident ensemble (owns its device memory until close())."""

    def __init__(self, ens: dict, t0: float = 0.0, stream=None):
        nb = np.ascontiguousarray(ens["n_body"], dtype=np.int32)
        self._mass = np.ascontiguousarray(ens["mass"], dtype=np.float64)
        pos = np.ascontiguousarray(ens["pos"], dtype=np.float64).reshape(-1, 3)
        vel = np.ascontiguousarray(ens["vel"], dtype=np.float64).reshape(-1, 3)
        self.n_body = nb
        self.n_sys = len(nb)
        self.n_bodies = int(nb.sum())
        h = _vp()
        _check(lib().swarm_create_ensemble(self.n_sys, nb.ctypes.data_as(_ip), _d(self._mass), _d(pos), _d(vel),
                                           float(t0), _stream_ptr(stream), C.byref(h)))
        self._h = h

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None):
            lib().swarm_destroy_ensemble(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- configuration
    def set_stop(self, ce_factor=0.0, eject_radius=0.0):
        _check(lib().swarm_set_stop(self._h, float(ce_factor), float(eject_radius)))

    def set_tolerance(self, eps):
        _check(lib().swarm_set_tolerance(self._h, float(eps)))

    def set_option(self, opt, value):
        _check(lib().swarm_set_option(self._h, int(opt), int(value)))

    # -- integration
    def integrate(self, t_end, integrator=HERMITE4, dt=None, sync=True):
        if dt is None:
            raise ValueError("dt is required")
        f = lib().swarm_integrate if sync else lib().swarm_integrate_async
        _check(f(self._h, float(t_end), int(integrator), float(dt)))

    def synchronize(self):
        _check(lib().swarm_synchronize(self._h))

    # -- state
    def set_state(self, pos=None, vel=None, time=None, status=None):
        p = None if pos is None else np.ascontiguousarray(pos, dtype=np.float64)
        v = None if vel is None else np.ascontiguousarray(vel, dtype=np.float64)
        t = None if time is None else np.ascontiguousarray(time, dtype=np.float64)
        s = None if status is None else np.ascontiguousarray(status, dtype=np.int32)
        _check(lib().swarm_set_state(self._h, _d(p), _d(v), _d(t), None if s is None else s.ctypes.data_as(_ip)))

    def state(self):
        pos = np.empty((self.n_bodies, 3))
        vel = np.empty((self.n_bodies, 3))
        tm = np.empty(self.n_sys)
        st = np.empty(self.n_sys, dtype=np.int32)
        _check(lib().swarm_query_state(self._h, _d(pos), _d(vel), _d(tm), st.ctypes.data_as(_ip)))
        return {"pos": pos, "vel": vel, "time": tm, "status": st}

    def state_into(self, pos=None, vel=None, time=None, status=None):
        """Host-pointer variant writing into caller-owned (e.g. pinned) numpy arrays."""
        _check(lib().swarm_query_state(self._h, _d(pos), _d(vel), _d(time),
                                       None if status is None else status.ctypes.data_as(_ip)))

    def set_state_dev(self, pos_t=None, vel_t=None, time_t=None, status_t=None):
        """Replace the state from device tensors (float64 [B,3], [B,3], [S]; int32 [S]),
        enqueued on the ensemble's stream."""
        ptr = lambda t: None if t is None else t.data_ptr()
        _check(lib().swarm_set_state_dev(self._h, ptr(pos_t), ptr(vel_t), ptr(time_t), ptr(status_t)))

    def state_dev(self, pos_t=None, vel_t=None, time_t=None, status_t=None):
        """Write the state into caller-owned torch CUDA tensors (float64 / int32), on the stream."""
        ptr = lambda t: None if t is None else t.data_ptr()
        _check(lib().swarm_query_state_dev(self._h, ptr(pos_t), ptr(vel_t), ptr(time_t), ptr(status_t)))

    def diagnostics(self):
        E = np.empty(self.n_sys)
        L = np.empty((self.n_sys, 3))
        _check(lib().swarm_query_diagnostics(self._h, _d(E), _d(L)))
        return E, L

    def log(self, sys_index, cap=65536):
        rec = np.empty((cap, 5))
        n = C.c_int32()
        _check(lib().swarm_query_log(self._h, int(sys_index), _d(rec), int(cap), C.byref(n)))
        return rec[: n.value].copy()

    def rv(self, los=(0.0, 0.0, 1.0)):
        """Radial velocity v_0 . los of every system's central body at the current state."""
        los = np.ascontiguousarray(los, dtype=np.float64)
        out = np.empty(self.n_sys)
        _check(lib().swarm_query_rv(self._h, _d(los), _d(out)))
        return out

    def observe_rv(self, t_obs, integrator, dt, los=(0.0, 0.0, 1.0)):
        """Integrate through the observation times; radial velocities [n_obs][n_sys]."""
        t_obs = np.ascontiguousarray(t_obs, dtype=np.float64)
        los = np.ascontiguousarray(los, dtype=np.float64)
        out = np.empty((len(t_obs), self.n_sys))
        _check(lib().swarm_observe_rv(self._h, _d(t_obs), len(t_obs), int(integrator), float(dt), _d(los), _d(out)))
        return out

    def stats(self):
        s = Stats()
        _check(lib().swarm_query_stats(self._h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in Stats._fields_}


def save_checkpoint(e: "Ensemble", path: str) -> None:
    """Write the ensemble's current state (masses, positions, velocities, times and
    statuses) to an .npz file; `load_checkpoint` + `Ensemble.resume` continue from it."""
    st = e.state()
    np.savez(path, n_body=e.n_body, mass=e._mass, pos=st["pos"], vel=st["vel"], time=st["time"], status=st["status"])


def load_checkpoint(path: str) -> dict:
    """Read a checkpoint written by `save_checkpoint` (the ics layout plus time, status)."""
    with np.load(path) as f:
        return {k: f[k] for k in ("n_body", "mass", "pos", "vel", "time", "status")}


def resume(ckpt: dict, stream=None) -> "Ensemble":
    """A new ensemble holding a checkpoint's state, times and statuses."""
    e = Ensemble(ckpt, stream=stream)
    e.set_state(time=ckpt["time"], status=ckpt["status"])
    return e


def fp64_peak(seconds=0.3, stream=None) -> float:
    out = C.c_double()
    _check(lib().swarm_fp64_peak(float(seconds), _stream_ptr(stream), C.byref(out)))
    return out.value


def tuner_choice(n, integrator, n_sys, stream=None):
    m, c = C.c_int32(), C.c_int32()
    _check(lib().swarm_tuner_choice(int(n), int(integrator), int(n_sys), _stream_ptr(stream), C.byref(m), C.byref(c)))
    return m.value, c.value


def tuner_load(path: str) -> None:
    """Load saved tuner choices (a missing file is not an error)."""
    _check(lib().swarm_tuner_load(path.encode()))


def tuner_save(path: str) -> None:
    _check(lib().swarm_tuner_save(path.encode()))


def version() -> str:
    return lib().swarm_version().decode()
