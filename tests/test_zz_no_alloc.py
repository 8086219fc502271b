"""The allocation-free entry point swarm_hermite_integrate_noalloc, called through the C
ABI on device buffers the caller owns (here torch tensors), must give the same results as
the regular entry point (swarm_create_ensemble + swarm_integrate) on two calls in a row.

It is for callers that cannot allocate device memory (a fixed memory budget or another
framework's pool, loops that must not synchronize on cudaMalloc, plugins restricted to
the buffers they are given); it keeps its working storage in a fixed device array.
This file is collected last so that a failure here never hides another test's result.
"""
import ctypes as C
import math

import numpy as np
import pytest

from gpu_util import TOL, per_system_errors
from paper_1208_1157_gb300 import ics

pytestmark = pytest.mark.gpu

DT = 2 * math.pi * 1e-3


def _fn():
    from paper_1208_1157_gb300 import swarm as S

    f = S.lib().swarm_hermite_integrate_noalloc
    vp = C.c_void_p
    f.argtypes = [C.c_int32, C.c_int32, C.c_int32, vp, vp, vp, vp, vp, C.c_double, C.c_double, C.c_double,
                  C.c_double, vp]
    f.restype = C.c_int
    return S, f


def _to_bin(ens, n, s_pad, torch):
    S = len(ens["n_body"])
    pos = ens["pos"].reshape(S, n, 3)
    vel = ens["vel"].reshape(S, n, 3)
    x = np.zeros((3, n, s_pad))
    v = np.zeros((3, n, s_pad))
    m = np.zeros((n, s_pad))
    x[:, :, :S] = pos.transpose(2, 1, 0)
    v[:, :, :S] = vel.transpose(2, 1, 0)
    m[:, :S] = ens["mass"].reshape(S, n).T
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return dev(x), dev(v), dev(m), torch.zeros(S, dtype=torch.float64, device="cuda"), \
        torch.zeros(S, dtype=torch.int32, device="cuda")


def _from_bin(x, v, t, st, S, n):
    xh, vh = x.cpu().numpy(), v.cpu().numpy()
    return {"pos": xh[:, :, :S].transpose(2, 1, 0).reshape(-1, 3), "vel": vh[:, :, :S].transpose(2, 1, 0).reshape(-1, 3),
            "time": t.cpu().numpy(), "status": st.cpu().numpy()}


@pytest.mark.parametrize("n", [3, 5])
def test_noalloc_matches_regular_entry_point_on_two_calls(n):
    torch = pytest.importorskip("torch")
    S_mod, f = _fn()
    S = 700 if n == 3 else 333
    ens = ics.three_body(S, seed=21) if n == 3 else ics.request_ensemble({"n_sys": S, "n": n, "seed": 77})
    s_pad = (S + 31) // 32 * 32
    x, v, m, t, st = _to_bin(ens, n, s_pad, torch)
    stream = torch.cuda.current_stream()
    ref = S_mod.Ensemble(ens, stream=stream)
    ref.set_stop(3.0, 100.0)
    for t_end in (300 * DT, 700 * DT):
        rc = f(n, S, s_pad, x.data_ptr(), v.data_ptr(), m.data_ptr(), t.data_ptr(), st.data_ptr(), t_end, DT, 3.0,
               100.0, stream.cuda_stream)
        assert rc == 0, S_mod.lib().swarm_last_error()
        torch.cuda.synchronize()
        got = _from_bin(x, v, t, st, S, n)
        ref.integrate(t_end, S_mod.HERMITE4, DT)
        want = ref.state()
        assert np.array_equal(got["status"], want["status"])
        np.testing.assert_allclose(got["time"], want["time"], rtol=1e-14, atol=0)
        ex, ev = per_system_errors(ens, got, want)
        assert ex.max() <= TOL and ev.max() <= TOL, (ex.max(), ev.max())
    ref.close()


def test_noalloc_rejects_oversized_ensembles():
    S_mod, f = _fn()
    dummy = C.c_void_p(16)
    # 65521 units of 32 systems exceed the fixed work list
    rc = f(3, 65521 * 32, 65521 * 32, dummy, dummy, dummy, dummy, dummy, 1.0, 0.1, 0.0, 0.0, None)
    assert rc == -1
    assert b"too large" in S_mod.lib().swarm_last_error()
