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


def test_noalloc_unpadded_rows_and_stopped_systems_untouched():
    """s_pad = n_sys (not a multiple of 32) and a few systems already stopped on entry:
    the stopped ones keep x, v, t and status bit for bit, the others match the regular
    entry point given the same statuses."""
    torch = pytest.importorskip("torch")
    S_mod, f = _fn()
    n, S = 4, 45
    ens = ics.request_ensemble({"n_sys": S, "n": n, "seed": 91})
    x, v, m, t, st = _to_bin(ens, n, S, torch)
    stopped = np.zeros(S, np.int32)
    stopped[::7] = S_mod.CLOSE_ENCOUNTER
    stopped[3] = S_mod.EJECTED
    st.copy_(torch.from_numpy(stopped))
    x0, v0 = x.clone(), v.clone()
    stream = torch.cuda.current_stream()
    ref = S_mod.Ensemble(ens, stream=stream)
    ref.set_stop(3.0, 100.0)
    ref.set_state(ens["pos"], ens["vel"], time=[0.0] * S, status=stopped)
    for t_end in (200 * DT, 450 * DT):
        rc = f(n, S, S, x.data_ptr(), v.data_ptr(), m.data_ptr(), t.data_ptr(), st.data_ptr(), t_end, DT, 3.0, 100.0,
               stream.cuda_stream)
        assert rc == 0, S_mod.lib().swarm_last_error()
        torch.cuda.synchronize()
        got = _from_bin(x, v, t, st, S, n)
        ref.integrate(t_end, S_mod.HERMITE4, DT)
        want = ref.state()
        assert np.array_equal(got["status"], want["status"])
        keep = stopped > S_mod.DONE
        assert np.array_equal(got["status"][keep], stopped[keep])
        assert np.all(got["time"][keep] == 0.0)
        assert torch.equal(x[:, :, torch.from_numpy(keep).cuda()], x0[:, :, torch.from_numpy(keep).cuda()])
        assert torch.equal(v[:, :, torch.from_numpy(keep).cuda()], v0[:, :, torch.from_numpy(keep).cuda()])
        run = ~keep
        np.testing.assert_allclose(got["time"][run], want["time"][run], rtol=1e-14, atol=0)
        ex, ev = per_system_errors(ens, got, want)
        assert ex.max() <= TOL and ev.max() <= TOL, (ex.max(), ev.max())
    ref.close()


def test_noalloc_marks_spans_beyond_the_step_limit():
    """A call asking more than 2e9 fixed steps of a system leaves it where it is with
    status SPAN_LIMIT (the times are on the device, so the check is per system there);
    already stopped systems keep their status."""
    torch = pytest.importorskip("torch")
    S_mod, f = _fn()
    n, S = 3, 40
    ens = ics.three_body(S, seed=5)
    x, v, m, t, st = _to_bin(ens, n, 64, torch)
    st[5] = S_mod.EJECTED
    x0, v0 = x.clone(), v.clone()
    stream = torch.cuda.current_stream()
    rc = f(n, S, 64, x.data_ptr(), v.data_ptr(), m.data_ptr(), t.data_ptr(), st.data_ptr(), 2.5e9 * DT, DT, 3.0,
           100.0, stream.cuda_stream)
    assert rc == 0, S_mod.lib().swarm_last_error()
    torch.cuda.synchronize()
    status = st.cpu().numpy()
    want = np.full(S, S_mod.SPAN_LIMIT, np.int32)
    want[5] = S_mod.EJECTED
    assert np.array_equal(status, want)
    assert torch.equal(x, x0) and torch.equal(v, v0)
    assert np.all(t.cpu().numpy() == 0.0)
