"""The C-ABI library: it loads, exports every entry point include/swarm.h declares, and
rejects bad arguments on the host before any device work (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1208_1157_gb300 import build as B
from paper_1208_1157_gb300 import ics

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def S():
    B.build()
    from paper_1208_1157_gb300 import swarm

    return swarm


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(swarm_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol(S):
    decl = declared_functions()
    assert len(decl) >= 15
    L = S.lib()
    missing = [n for n in sorted(decl) if not hasattr(L, n)]
    assert not missing, missing
    assert set(S.EXPORTS) <= decl


def test_version_and_error_string(S):
    assert "sm_103a" in S.version()
    assert isinstance(S.lib().swarm_last_error(), bytes)


def _create(S, ens, t0=0.0):
    L = S.lib()
    h = C.c_void_p()
    nb = np.ascontiguousarray(ens["n_body"], dtype=np.int32)
    d = lambda a: np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(C.POINTER(C.c_double))
    rc = L.swarm_create_ensemble(len(nb), nb.ctypes.data_as(C.POINTER(C.c_int32)), d(ens["mass"]), d(ens["pos"]),
                                 d(ens["vel"]), t0, None, C.byref(h))
    return rc, h


@pytest.mark.parametrize("case", ["n_too_small", "n_too_large", "nan_pos", "zero_mass", "inf_t0", "empty"])
def test_create_rejects_bad_input_on_host(S, case):
    ens = ics.three_body(4, seed=1)
    t0 = 0.0
    if case == "n_too_small":
        ens = {"n_body": np.array([1]), "mass": np.array([1.0]), "pos": np.zeros((1, 3)), "vel": np.zeros((1, 3))}
    elif case == "n_too_large":
        ens = {"n_body": np.array([33]), "mass": np.ones(33), "pos": np.arange(99.0).reshape(33, 3), "vel": np.zeros((33, 3))}
    elif case == "nan_pos":
        ens["pos"][4, 1] = np.nan
    elif case == "zero_mass":
        ens["mass"][2] = 0.0
    elif case == "inf_t0":
        t0 = float("inf")
    elif case == "empty":
        ens = {"n_body": np.zeros(0, np.int32), "mass": np.zeros(0), "pos": np.zeros((0, 3)), "vel": np.zeros((0, 3))}
    rc, h = _create(S, ens, t0)
    assert rc == S.EINVAL and not h.value
    assert len(S.lib().swarm_last_error()) > 0


def test_null_handles_are_rejected(S):
    L = S.lib()
    assert L.swarm_integrate(None, 1.0, 1, 0.1) == S.EINVAL
    assert L.swarm_set_option(None, 1, 0) == S.EINVAL
    assert L.swarm_query_state(None, None, None, None, None) == S.EINVAL
    assert L.swarm_ensemble_size(None) == 0
    L.swarm_destroy_ensemble(None)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import importlib

    import paper_1208_1157_gb300.swarm as sw

    mod = importlib.reload(sw)
    monkeypatch.setattr(mod, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(mod, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        mod.lib()
    importlib.reload(sw)
