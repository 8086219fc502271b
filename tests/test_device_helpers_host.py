"""Device helpers compiled from the kernel sources as host code (no GPU: gcc and the
source text), checked in 30-50 digit arithmetic: the Stumpff functions of the Kepler drift
(csrc/mvs_impl.cuh, `stumpff23`: power series to |z| <= 0.25, argument quartering and the
doubling relations beyond) against the closed forms
    c2(z) = (1 - cos sqrt z) / z,  c3(z) = (sqrt z - sin sqrt z) / z^(3/2)
(cosh / sinh for z < 0), and the Runge-Kutta step control's e^(-1/10)
(csrc/rkck_impl.cuh, `inv_tenth_root`)."""
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1208_1157_gb300", "csrc",
                   "mvs_impl.cuh")


@pytest.fixture(scope="module")
def stumpff_exe(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    text = open(SRC).read()
    fn = re.search(r"__device__ __forceinline__ void stumpff23\(double z, double &c2, double &c3\) \{.*?\n\}\n",
                   text, re.S).group(0).replace("__device__ __forceinline__ ", "static ")
    prog = ("#include <cmath>\n#include <cstdio>\n#include <cstdlib>\nusing std::fabs; using std::fma;\n" + fn +
            "int main(int argc, char **argv) {\n"
            "  double z;\n"
            "  while (scanf(\"%lf\", &z) == 1) { double c2, c3; stumpff23(z, c2, c3); printf(\"%.17g %.17g\\n\", c2, c3); }\n"
            "  return 0;\n}\n")
    d = tmp_path_factory.mktemp("stumpff")
    (d / "s.cpp").write_text(prog)
    exe = d / "s"
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-o", str(exe), str(d / "s.cpp")], check=True)
    return exe


def run(exe, zs):
    out = subprocess.run([str(exe)], input="\n".join(repr(float(z)) for z in zs), capture_output=True, text=True,
                         check=True).stdout.split()
    v = np.array([float(t) for t in out]).reshape(-1, 2)
    return v[:, 0], v[:, 1]


def exact(z):
    mp.mp.dps = 50
    z = mp.mpf(z)
    if abs(z) < mp.mpf("1e-8"):  # the closed forms cancel: their series
        return (mp.mpf(1) / 2 - z / 24 + z * z / 720 - z ** 3 / 40320,
                mp.mpf(1) / 6 - z / 120 + z * z / 5040 - z ** 3 / 362880)
    if z > 0:
        s = mp.sqrt(z)
        return (1 - mp.cos(s)) / z, (s - mp.sin(s)) / (s ** 3)
    s = mp.sqrt(-z)
    return (mp.cosh(s) - 1) / (-z), (mp.sinh(s) - s) / (s ** 3)


def rel_err(exe, zs):
    c2, c3 = run(exe, zs)
    e2 = max(abs(float((mp.mpf(a) - exact(z)[0]) / exact(z)[0])) for a, z in zip(c2, zs))
    e3 = max(abs(float((mp.mpf(b) - exact(z)[1]) / exact(z)[1])) for b, z in zip(c3, zs))
    return e2, e3


def test_series_range(stumpff_exe):
    # the range the Kepler drift of 1/20-orbit steps meets: the series alone
    zs = np.concatenate([np.linspace(-0.25, 0.25, 201), [0.0, 1e-300, -1e-12, 0.099, 0.25, -0.25]])
    e2, e3 = rel_err(stumpff_exe, zs)
    assert e2 <= 3e-16 and e3 <= 3e-16, (e2, e3)


def test_quartering_and_doubling(stumpff_exe):
    # elliptic arguments up to (2 pi)^2 (a whole orbit) and hyperbolic ones; near
    # z = (2 pi)^2, c2 is small against the terms of the doubling (7e-14 relative there)
    zs = np.concatenate([np.linspace(0.26, 39.0, 97), -np.linspace(0.26, 30.0, 60)])
    e2, e3 = rel_err(stumpff_exe, zs)
    assert e2 <= 3e-13 and e3 <= 3e-13, (e2, e3)


def test_universal_identity(stumpff_exe):
    # c0 = 1 - z c2 and c1 = 1 - z c3 satisfy c0^2 + z c1^2 = 1 (cos^2 + sin^2 = 1)
    zs = np.linspace(-20.0, 39.0, 119)
    c2, c3 = run(stumpff_exe, zs)
    c0 = 1 - zs * c2
    c1 = 1 - zs * c3
    assert np.max(np.abs(c0 * c0 + zs * c1 * c1 - 1.0) / np.maximum(1.0, c0 * c0)) <= 1e-12


RK = os.path.join(os.path.dirname(SRC), "rkck_impl.cuh")


def test_step_control_root_host():
    # inv_tenth_root (the Runge-Kutta step control's err^(-1/5) from the squared error),
    # compiled from the kernel source as host code: e^(-1/10) to ~1e-12 over [1e-30, 1e30]
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    import tempfile
    text = open(RK).read()
    fn = re.search(r"__device__ __forceinline__ double inv_tenth_root\(double e\) \{.*?\n\}\n", text,
                   re.S).group(0).replace("__device__ __forceinline__ ", "static ")
    prog = ("#include <cmath>\n#include <cstdio>\nusing std::fma; using std::exp2f; using std::log2f;\n" + fn +
            "int main() { double e; while (scanf(\"%lf\", &e) == 1) printf(\"%.17g\\n\", inv_tenth_root(e)); return 0; }\n")
    d = tempfile.mkdtemp()
    with open(os.path.join(d, "r.cpp"), "w") as f:
        f.write(prog)
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-o", os.path.join(d, "r"), os.path.join(d, "r.cpp")],
                   check=True)
    es = np.logspace(-30, 30, 601)
    out = subprocess.run([os.path.join(d, "r")], input="\n".join(repr(float(e)) for e in es), capture_output=True,
                         text=True, check=True).stdout.split()
    mp.mp.dps = 30
    err = max(abs(float((mp.mpf(y) - mp.power(mp.mpf(e), mp.mpf(-1) / 10)) / mp.power(mp.mpf(e), mp.mpf(-1) / 10)))
              for y, e in zip(out, es))
    assert err <= 5e-12, err
