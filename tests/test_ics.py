"""The seeded input generator: determinism, frame, and the stated distributions."""
import math

import numpy as np

from paper_1208_1157_gb300 import ics


def _astro(ens, s):
    sub = ics.subset(ens, [s])
    return sub["mass"], sub["pos"] - sub["pos"][0], sub["vel"] - sub["vel"][0]


def test_deterministic_and_counter_based():
    a = ics.three_body(64, seed=1)
    b = ics.three_body(64, seed=1)
    for k in a:
        assert np.array_equal(a[k], b[k])
    # system s does not depend on how many systems were drawn
    c = ics.three_body(16, seed=1)
    assert np.array_equal(c["pos"], a["pos"][: 16 * 3])
    d = ics.three_body(64, seed=2)
    assert not np.array_equal(d["pos"], a["pos"])


def test_uniform_range_and_mean():
    u = ics.uniform(7, np.arange(200000), 3)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 3e-3


def test_barycentric_frame():
    for ens in (ics.three_body(32, 1), ics.ragged(32, 3), ics.mvs_compact(16, 4)):
        offs = np.concatenate([[0], np.cumsum(ens["n_body"])])
        for s in range(len(ens["n_body"])):
            sl = slice(offs[s], offs[s + 1])
            m = ens["mass"][sl]
            assert np.max(np.abs((m[:, None] * ens["pos"][sl]).sum(0))) < 1e-15
            assert np.max(np.abs((m[:, None] * ens["vel"][sl]).sum(0))) < 1e-15


def test_three_body_distributions():
    ens = ics.three_body(2000, seed=1)
    for s in range(0, 2000, 97):
        m, r, v = _astro(ens, s)
        assert m[0] == 1.0 and 1e-5 <= m[1] <= 1e-3 and 1e-5 <= m[2] <= 1e-3
        for j, (lo, hi) in zip((1, 2), ((1.0, 1.0), (1.6, 3.0))):
            mu = 1.0 + m[j]
            a = 1.0 / (2.0 / np.linalg.norm(r[j]) - v[j] @ v[j] / mu)
            h = np.cross(r[j], v[j])
            e = math.sqrt(max(0.0, 1.0 - (h @ h) / (mu * a)))
            inc = math.acos(h[2] / np.linalg.norm(h))
            assert lo - 1e-9 <= a <= hi + 1e-9
            assert e <= 0.05 + 1e-9 and inc <= 0.01 + 1e-9


def test_ragged_and_compact_shapes():
    r = ics.ragged(4000, seed=3)
    assert r["n_body"].min() == 3 and r["n_body"].max() == 15
    counts = np.bincount(r["n_body"], minlength=16)[3:]
    assert counts.min() > 200  # roughly uniform over 13 values
    c = ics.mvs_compact(200, seed=4)
    assert np.all(c["n_body"] == 8)
    offs = np.concatenate([[0], np.cumsum(c["n_body"])])
    for s in range(200):
        x = c["pos"][offs[s]:offs[s + 1]]
        assert np.max(np.linalg.norm(x[1:] - x[0], axis=1)) < 50.0


def test_serving_trace():
    tr = ics.serving_trace(512, seed=5)
    arr = np.array([q["arrival_s"] for q in tr])
    assert np.all(np.diff(arr) >= 0) and arr[0] == 0.0
    assert 1.5 < arr[-1] < 4.0  # 511 gaps of mean 5 ms
    sizes = np.array([q["n_sys"] for q in tr])
    assert sizes.min() >= 1 and sizes.max() <= 4096
    assert 250 < sizes.mean() < 800
    e = ics.request_ensemble(tr[3])
    assert len(e["n_body"]) == tr[3]["n_sys"]
