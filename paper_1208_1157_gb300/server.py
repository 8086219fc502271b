"""ctypes binding of the continuous-batching server (swarm_server_* in include/swarm.h)
and a driver that replays a request trace in wall-clock time.
"""
from __future__ import annotations

import ctypes as C
import time

import numpy as np

from . import ics
from . import swarm as S

REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_CANCELLED = 0, 1, 2, 3


class Config(C.Structure):
    _fields_ = [("slots_per_pool", C.c_int32), ("quantum_steps", C.c_int32), ("hermite_dt", C.c_double),
                ("mvs_dt", C.c_double), ("ce_hill_factor", C.c_double), ("eject_radius", C.c_double),
                ("device_bytes", C.c_int64)]


class Stats(C.Structure):
    _fields_ = [(f, C.c_int64) for f in ("submitted", "admitted", "completed", "queued", "occupied_slots",
                                         "pool_slots", "device_bytes", "quanta", "system_steps", "pair_evaluations")] + \
               [("kernel_ms", C.c_double), ("cancelled", C.c_int64)]


_decl = False


def _lib():
    global _decl
    L = S.lib()
    if not _decl:
        vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32)
        L.swarm_server_create.argtypes = [C.POINTER(Config), vp, C.POINTER(vp)]
        L.swarm_server_submit.argtypes = [vp, C.c_int32, C.c_int32, dp, dp, dp, C.c_double, C.c_double, C.c_int,
                                          C.POINTER(C.c_int64)]
        L.swarm_server_step.argtypes = [vp, ip]
        L.swarm_server_poll.argtypes = [vp, C.c_int64, ip, dp, dp, dp, ip, dp]
        L.swarm_server_release.argtypes = [vp, C.c_int64]
        L.swarm_server_cancel.argtypes = [vp, C.c_int64]
        L.swarm_server_query.argtypes = [vp, C.POINTER(Stats)]
        L.swarm_server_destroy.argtypes = [vp]
        L.swarm_server_destroy.restype = None
        _decl = True
    return L


class Server:
    def __init__(self, slots_per_pool=8192, quantum_steps=200, hermite_dt=2 * np.pi * 1e-3, mvs_dt=2 * np.pi / 20,
                 ce_hill_factor=3.0, eject_radius=100.0, device_bytes=0, stream=None):
        cfg = Config(slots_per_pool, quantum_steps, hermite_dt, mvs_dt, ce_hill_factor, eject_radius, device_bytes)
        h = C.c_void_p()
        S._check(_lib().swarm_server_create(C.byref(cfg), S._stream_ptr(stream), C.byref(h)))
        self._h = h
        self.cfg = cfg

    def close(self):
        if getattr(self, "_h", None):
            _lib().swarm_server_destroy(self._h)
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

    def submit(self, ens: dict, t_end: float, integrator: int, t0: float = 0.0) -> int:
        nb = np.asarray(ens["n_body"])
        n = int(nb[0])
        assert np.all(nb == n), "a request holds systems of one body count"
        d = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        m, p, v = d(ens["mass"]), d(ens["pos"]), d(ens["vel"])
        rid = C.c_int64()
        S._check(_lib().swarm_server_submit(self._h, len(nb), n, S._d(m), S._d(p), S._d(v), float(t0), float(t_end),
                                            int(integrator), C.byref(rid)))
        return rid.value

    def step(self) -> int:
        k = C.c_int32()
        S._check(_lib().swarm_server_step(self._h, C.byref(k)))
        return k.value

    def poll(self, rid: int, n_sys: int = 0, n: int = 0):
        st = C.c_int32()
        if n_sys:
            pos = np.empty((n_sys * n, 3))
            vel = np.empty((n_sys * n, 3))
            tm = np.empty(n_sys)
            ss = np.empty(n_sys, dtype=np.int32)
            lat = C.c_double()
            S._check(_lib().swarm_server_poll(self._h, rid, C.byref(st), S._d(pos), S._d(vel), S._d(tm),
                                              ss.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(lat)))
            if st.value == REQ_DONE:
                return st.value, {"pos": pos, "vel": vel, "time": tm, "status": ss, "latency_s": lat.value}
            return st.value, None
        S._check(_lib().swarm_server_poll(self._h, rid, C.byref(st), None, None, None, None, None))
        return st.value, None

    def cancel(self, rid: int):
        S._check(_lib().swarm_server_cancel(self._h, rid))

    def release(self, rid: int):
        S._check(_lib().swarm_server_release(self._h, rid))

    def stats(self) -> dict:
        s = Stats()
        S._check(_lib().swarm_server_query(self._h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in Stats._fields_}


def replay(server: Server, trace: list, ensembles: list | None = None, collect: bool = False, max_wall_s: float = 600.0):
    """Submit each request of `trace` at its arrival time (wall clock from now) while
    stepping the server continuously; returns per-request latency and results."""
    if ensembles is None:
        ensembles = [ics.request_ensemble(q) for q in trace]
    integ = {1: S.HERMITE4, 2: S.MVS_DH, 3: S.MVS_JACOBI}
    ids, done = {}, {}
    occupancy = []
    t_start = time.perf_counter()
    nxt = 0
    while len(done) < len(trace):
        now = time.perf_counter() - t_start
        if now > max_wall_s:
            raise TimeoutError(f"trace not drained after {max_wall_s} s ({len(done)}/{len(trace)} done)")
        while nxt < len(trace) and trace[nxt]["arrival_s"] <= now:
            q = trace[nxt]
            ids[server.submit(ensembles[nxt], q["t_end"], integ[q["integrator"]])] = nxt
            nxt += 1
        if not ids or len(done) == len(ids):
            if nxt < len(trace):
                time.sleep(min(0.001, max(0.0, trace[nxt]["arrival_s"] - now)))
            continue
        k = server.step()
        st = server.stats()
        occupancy.append((time.perf_counter() - t_start, st["occupied_slots"], st["queued"]))
        if k:
            for rid, r in list(ids.items()):
                if r in done:
                    continue
                q = trace[r]
                state, res = server.poll(rid, q["n_sys"], q["n"])
                if state == REQ_DONE:
                    done[r] = res if collect else {"latency_s": res["latency_s"]}
                    server.release(rid)
    wall = time.perf_counter() - t_start
    return {"done": done, "wall_s": wall, "occupancy": occupancy, "stats": server.stats()}
