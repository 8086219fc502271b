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


HOST_SHIMS = (
    "#include <cmath>\n#include <cstdio>\n#include <cstdlib>\n#include <cstring>\n"
    "using std::fabs; using std::fma; using std::sqrt; using std::fmax;\n"
    "#define __device__\n#define __forceinline__ inline\n#define __noinline__\n"
    "static inline int __double2hiint(double a) { long long b; std::memcpy(&b, &a, 8); return (int)(b >> 32); }\n"
    "static inline long long __double_as_longlong(double a) { long long b; std::memcpy(&b, &a, 8); return b; }\n"
    "static inline bool __all_sync(unsigned, bool p) { return p; }\n"
    "static inline double rsqrt(double x) { return 1.0 / std::sqrt(x); }\n")


def common_helpers():
    """The scalar helpers of csrc/common.cuh the Kepler drift and the Stumpff functions use
    (F64k forms, integer-pipe compares, the refined reciprocal), as host code; the
    reciprocal's hardware seed (inline PTX) becomes an exact 1/d."""
    common = open(COMMON).read()
    f64k = re.search(r"struct F64k \{.*?kadd\(const F64k &k, double a, double b\) \{ return fma\(a, k.one, b\); \}\n",
                     common, re.S).group(0)
    out = [f64k]
    for sig in (r"bool nonneg_lt\(double a, double b\)", r"bool abs_below_pow2\(double a, int e\)",
                r"double rcp_newton\(const F64k &k, double d\)"):
        out.append(re.search(r"__device__ __forceinline__ " + sig + r" \{.*?\n\}\n", common, re.S).group(0))
    text = "".join(out)
    seed = re.search(r'  asm\("rcp\.approx\.ftz\.f64 %0, %1;" : "=d"\(r\) : "d"\(d\)\);\n', text)
    assert seed, "the reciprocal seed is not in common.cuh"
    return text.replace(seed.group(0), "  r = 1.0 / d;\n")


def build_stumpff(d):
    """Host build of the kernel's stumpff23 (from SRC) in directory d."""
    text = open(SRC).read()
    fn = re.search(r"__device__ __forceinline__ void stumpff23\(double z, double &c2, double &c3\) \{.*?\n\}\n",
                   text, re.S).group(0)
    prog = (HOST_SHIMS + "namespace swarm {\n" + common_helpers() + fn + "}\nusing swarm::stumpff23;\n" +
            "int main(int argc, char **argv) {\n"
            "  double z;\n"
            "  while (scanf(\"%lf\", &z) == 1) { double c2, c3; stumpff23(z, c2, c3); printf(\"%.17g %.17g\\n\", c2, c3); }\n"
            "  return 0;\n}\n")
    with open(os.path.join(d, "s.cpp"), "w") as f:
        f.write(prog)
    exe = os.path.join(d, "s")
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-o", exe, os.path.join(d, "s.cpp")], check=True)
    return exe


@pytest.fixture(scope="module")
def stumpff_exe(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    return build_stumpff(str(tmp_path_factory.mktemp("stumpff")))


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


def check_series_range(exe):
    # the range the Kepler drift of 1/20-orbit steps meets: the series alone
    zs = np.concatenate([np.linspace(-0.25, 0.25, 201), [0.0, 1e-300, -1e-12, 0.099, 0.25, -0.25]])
    e2, e3 = rel_err(exe, zs)
    assert e2 <= 3e-16 and e3 <= 3e-16, (e2, e3)


def check_quartering_and_doubling(exe):
    # elliptic arguments up to (2 pi)^2 (a whole orbit) and hyperbolic ones; near
    # z = (2 pi)^2, c2 is small against the terms of the doubling (7e-14 relative there)
    zs = np.concatenate([np.linspace(0.26, 39.0, 97), -np.linspace(0.26, 30.0, 60)])
    e2, e3 = rel_err(exe, zs)
    assert e2 <= 3e-13 and e3 <= 3e-13, (e2, e3)


def test_series_range(stumpff_exe):
    check_series_range(stumpff_exe)


def test_quartering_and_doubling(stumpff_exe):
    check_quartering_and_doubling(stumpff_exe)


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


COMMON = os.path.join(os.path.dirname(SRC), "common.cuh")

KEPLER_MAIN = r"""
int main() {
  // per line: mu h steps rx ry rz vx vy vz; prints the state after every step and the
  // Newton iterations of that step
  double mu, h, r[3], v[3];
  int steps;
  const swarm::F64k k = {0.0, -1.0, 1.0};
  while (scanf("%lf %lf %d %lf %lf %lf %lf %lf %lf", &mu, &h, &steps, &r[0], &r[1], &r[2], &v[0], &v[1], &v[2]) == 9) {
    const swarm::KepConst K = swarm::kep_const(mu);
    double rq = 1.0;
    for (int s = 0; s < steps; s++) {
      int it = 0;
      const bool ok = swarm::kepler_drift<false>(k, true, K, r, v, h, it, rq);
      printf("%d %d %.17g %.17g %.17g %.17g %.17g %.17g\n", ok ? 1 : 0, it, r[0], r[1], r[2], v[0], v[1], v[2]);
    }
  }
  return 0;
}
"""


def build_kepler(d):
    """Host build of the kernel's kepler_drift (from COMMON and SRC) in directory d."""
    mvs = open(SRC).read()
    stumpff = re.search(r"__device__ __forceinline__ void stumpff23\(double z, double &c2, double &c3\) \{.*?\n\}\n",
                        mvs, re.S).group(0)
    # up to the replica-shared form of the drift (warp shuffles; its bits are the plain
    # drift's, checked on the GPU against a system integrated alone)
    kep = mvs[mvs.index("struct KepConst {"):mvs.index("// ---------------------------------------------------------------- drift shared by replicas")]
    prog = HOST_SHIMS + "namespace swarm {\n" + common_helpers() + stumpff + kep + "}\n" + KEPLER_MAIN
    with open(os.path.join(d, "k.cpp"), "w") as f:
        f.write(prog)
    exe = os.path.join(d, "k")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-o", exe, os.path.join(d, "k.cpp")], check=True)
    return exe


@pytest.fixture(scope="module")
def kepler_exe(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    return build_kepler(str(tmp_path_factory.mktemp("kepler")))


def kepler_exact(mu, r0, v0, t):
    """Two-body state after time t: Kepler's equation solved in 40-digit arithmetic."""
    mp.mp.dps = 40
    r0 = [mp.mpf(x) for x in r0]
    v0 = [mp.mpf(x) for x in v0]
    mu = mp.mpf(mu)
    t = mp.mpf(t)
    rn = mp.sqrt(sum(x * x for x in r0))
    v2 = sum(x * x for x in v0)
    a = 1 / (2 / rn - v2 / mu)
    rv = sum(x * y for x, y in zip(r0, v0))
    if a > 0:
        n = mp.sqrt(mu / a ** 3)
        ecosE, esinE = 1 - rn / a, rv / mp.sqrt(mu * a)
        # solve for the change of eccentric anomaly dE: n t = dE - ecosE sin dE + esinE (1 - cos dE)
        dE = mp.findroot(lambda x: x - ecosE * mp.sin(x) + esinE * (1 - mp.cos(x)) - n * t, n * t)
        f = 1 - a / rn * (1 - mp.cos(dE))
        g = t - (dE - mp.sin(dE)) / n
        r = [f * x + g * y for x, y in zip(r0, v0)]
        rr = mp.sqrt(sum(x * x for x in r))
        fd = -mp.sqrt(mu * a) / (rr * rn) * mp.sin(dE)
        gd = 1 - a / rr * (1 - mp.cos(dE))
    else:
        an = -a
        n = mp.sqrt(mu / an ** 3)
        ecoshF, esinhF = 1 + rn / an, rv / mp.sqrt(mu * an)
        dF = mp.findroot(lambda x: -x + ecoshF * mp.sinh(x) + esinhF * (mp.cosh(x) - 1) - n * t, mp.asinh(n * t))
        f = 1 - an / rn * (mp.cosh(dF) - 1)
        g = t - (mp.sinh(dF) - dF) / n
        r = [f * x + g * y for x, y in zip(r0, v0)]
        rr = mp.sqrt(sum(x * x for x in r))
        fd = -mp.sqrt(mu * an) / (rr * rn) * mp.sinh(dF)
        gd = 1 - an / rr * (mp.cosh(dF) - 1)
    v = [fd * x + gd * y for x, y in zip(r0, v0)]
    return [float(x) for x in r], [float(x) for x in v]


def drift_run(exe, mu, h, steps, r, v):
    line = " ".join([repr(float(mu)), repr(float(h)), str(int(steps))] + [repr(float(x)) for x in [*r, *v]])
    out = subprocess.run([str(exe)], input=line, capture_output=True, text=True, check=True).stdout.split("\n")
    rows = [list(map(float, l.split())) for l in out if l.strip()]
    return np.array(rows)


def check_kepler_elliptic(kepler_exe, e):
    # the kernel's drift (fourth-order Taylor start, one Halley step, error-bound stop,
    # Taylor finalize) over 60 steps of 1/20 orbit against Kepler's equation: the state to
    # 1e-13; a single iteration per step for e <= 0.05, at most two for e <= 0.3
    mu, a = 1.0 + 1e-3, 1.3
    r0 = [a * (1 - e), 0.0, 0.01]
    v0 = [0.0, float(np.sqrt(mu * (1 + e) / (a * (1 - e)))), 0.002]
    T = 2 * np.pi * np.sqrt(a ** 3 / mu)
    h = T / 20
    rows = drift_run(kepler_exe, mu, h, 60, r0, v0)
    assert np.all(rows[:, 0] == 1)
    for s in (0, 9, 19, 39, 59):
        rx, vx = kepler_exact(mu, r0, v0, h * (s + 1))
        assert np.max(np.abs(rows[s, 2:5] - rx)) <= 1e-13 * np.max(np.abs(rx)) * (s + 1)
        assert np.max(np.abs(rows[s, 5:8] - vx)) <= 1e-13 * np.max(np.abs(vx)) * (s + 1)
    if e <= 0.05:
        assert np.all(rows[:, 1] == 1), rows[:, 1]
    if e <= 0.3:
        assert rows[:, 1].max() <= 2, rows[:, 1]


@pytest.mark.parametrize("e", [0.0, 0.05, 0.3, 0.9])
def test_kepler_drift_elliptic_host(kepler_exe, e):
    check_kepler_elliptic(kepler_exe, e)


def test_kepler_drift_hyperbolic_host(kepler_exe):
    mu = 1.0
    r0 = [1.0, 0.0, 0.0]
    v0 = [0.0, 1.8, 0.1]  # v^2 > 2 mu / r: unbound
    h = 0.05
    rows = drift_run(kepler_exe, mu, h, 40, r0, v0)
    assert np.all(rows[:, 0] == 1)
    rx, vx = kepler_exact(mu, r0, v0, h * 40)
    assert np.max(np.abs(rows[-1, 2:5] - rx)) <= 1e-12 * np.max(np.abs(rx))
    assert np.max(np.abs(rows[-1, 5:8] - vx)) <= 1e-12 * np.max(np.abs(vx))


HERMITE = os.path.join(os.path.dirname(SRC), "hermite.cuh")

REL_MAIN = r"""
#include <random>
using namespace swarm;
static double relmax(const double (&a)[3][3], const double (&b)[3][3], int i0) {
  double e = 0.0, s = 0.0;
  for (int i = i0; i < 3; i++) for (int c = 0; c < 3; c++) { e = fmax(e, fabs(a[i][c] - b[i][c])); s = fmax(s, fabs(b[i][c])); }
  return e / s;
}
int main() {
  const F64k k = {0.0, -1.0, 1.0};
  std::mt19937_64 g(7);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  double worst_acc = 0, worst_jerk = 0, worst_round = 0, worst_cached = 0, worst_fallback = 0;
  for (int trial = 0; trial < 2000; trial++) {
    double m[3] = {1.0, 1e-3 * (1.5 + U(g)), 1e-3 * (1.5 + U(g))};
    if (trial % 4 == 0) { m[1] = 0.5 + 0.3 * U(g); m[2] = 0.5 + 0.3 * U(g); }  // comparable masses
    double x[3][3], v[3][3];
    for (int i = 0; i < 3; i++) for (int c = 0; c < 3; c++) { x[i][c] = (i ? 1.5 * i : 0.0) * (c == 0) + 0.4 * U(g); v[i][c] = 0.5 * U(g); }
    double a[3][3], j[3][3], q2[3], d2[3][3];
    spl_accjerk<3>(k, x, v, m, a, j, q2, d2);               // inertial
    double X[3][3], V[3][3], Minv, Xc[3], Vc[3];
    for (int i = 0; i < 3; i++) for (int c = 0; c < 3; c++) { X[i][c] = x[i][c]; V[i][c] = v[i][c]; }
    spl_to_rel<3>(m, X, V, Minv, Xc, Vc);
    double A[3][3], J[3][3];
    spl_accjerk_rel<3>(k, X, V, m, A, J, q2, d2);
    double ai[3][3], ji[3][3];                               // inertial from relative
    for (int c = 0; c < 3; c++) { ai[0][c] = A[0][c]; ji[0][c] = J[0][c];
      for (int i = 1; i < 3; i++) { ai[i][c] = A[i][c] + A[0][c]; ji[i][c] = J[i][c] + J[0][c]; } }
    worst_acc = fmax(worst_acc, relmax(ai, a, 0));
    worst_jerk = fmax(worst_jerk, relmax(ji, j, 0));
    double xo[3][3], vo[3][3];
    spl_from_rel<3>(m, X, V, Minv, Xc, Vc, xo, vo);
    worst_round = fmax(worst_round, fmax(relmax(xo, x, 0), relmax(vo, v, 0)));
    // cached 1/|d|: fill at X, evaluate at a corrector-sized move and at a large one
    for (int big = 0; big < 2; big++) {
      RhoCache<3> rc;
      double A1[3][3], J1[3][3], A2[3][3], J2[3][3], Y[3][3];
      spl_accjerk_rel_cached<3, true>(k, X, V, m, A1, J1, q2, d2, rc);
      for (int i = 1; i < 3; i++) for (int c = 0; c < 3; c++) Y[i][c] = X[i][c] * (1.0 + (big ? 1e-3 : 1e-10) * U(g));
      spl_accjerk_rel_cached<3, false>(k, Y, V, m, A2, J2, q2, d2, rc);
      spl_accjerk_rel<3>(k, Y, V, m, A1, J1, q2, d2);        // reference: rsqrt
      double e = fmax(relmax(A2, A1, 1), relmax(J2, J1, 1));
      if (big) worst_fallback = fmax(worst_fallback, e); else worst_cached = fmax(worst_cached, e);
    }
  }
  printf("%.3e %.3e %.3e %.3e %.3e\n", worst_acc, worst_jerk, worst_round, worst_cached, worst_fallback);
  return 0;
}
"""


def test_star_relative_evaluation_host():
    # the system-per-lane Hermite kernel's relative-coordinate evaluation (spl_accjerk_rel,
    # its cached-1/|d| variant and the frame maps), compiled as host code: A_k + A_0 and
    # J_k + J_0 equal the inertial a_k, j_k of the same kernel file's inertial evaluation,
    # the frame maps round-trip, and the series-refined 1/|d| (corrector-sized moves) and
    # its rsqrt fallback (large moves) agree with rsqrt
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    import tempfile
    common = open(COMMON).read()
    herm = open(HERMITE).read()
    f64k = re.search(r"struct F64k \{.*?kadd\(const F64k &k, double a, double b\) \{ return fma\(a, k.one, b\); \}\n",
                     common, re.S).group(0)
    pair = re.search(r"__device__ __forceinline__ void pair_geom\(.*?\n\}\n", herm, re.S).group(0)
    inert = re.search(r"template <int N>\n__device__ __forceinline__ void spl_accjerk\(.*?\n\}\n", herm, re.S).group(0)
    rel = herm[herm.index("// Coordinates relative to body 0"):
               herm.index("template <int N>\n__device__ __forceinline__ void spl_energy(")]
    prog = ("#include <cmath>\n#include <cstdio>\n#include <cstring>\n"
            "using std::fabs; using std::fma; using std::sqrt; using std::fmax;\n"
            "#define __device__\n#define __forceinline__ inline\n#define __noinline__\n"
            "static inline double rsqrt(double x) { return 1.0 / std::sqrt(x); }\n"
            "static inline int __double2hiint(double x) { long long b; std::memcpy(&b, &x, 8); return (int)(b >> 32); }\n"
            "namespace swarm {\n" + f64k + pair + inert + rel + "}\n" + REL_MAIN)
    d = tempfile.mkdtemp()
    with open(os.path.join(d, "r.cpp"), "w") as f:
        f.write(prog)
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-Wno-unknown-pragmas", "-o",
                    os.path.join(d, "r"), os.path.join(d, "r.cpp")], check=True)
    acc, jerk, rnd, cached, fallback = map(float, subprocess.run([os.path.join(d, "r")], capture_output=True,
                                                                 text=True, check=True).stdout.split())
    print("relative-frame evaluation:", acc, jerk, rnd, cached, fallback)
    assert acc <= 1e-14 and jerk <= 1e-14, (acc, jerk)
    assert rnd <= 1e-15, rnd
    # the series and rsqrt round differently: a few units in the last place of 1/|d|,
    # relative to the largest acceleration or jerk of the system
    assert cached <= 1e-14 and fallback <= 1e-15, (cached, fallback)


RK_MAIN = r"""
using namespace swarm;
int main() {
  // per line: m0 m1 m2, x (9), v (9), h; prints the 5th-order x, v and the error vectors
  // (position, velocity) of all bodies in inertial coordinates
  const F64k k = {0.0, -1.0, 1.0};
  double m[3], x[3][3], v[3][3], h;
  while (scanf("%lf %lf %lf", &m[0], &m[1], &m[2]) == 3) {
    for (int i = 0; i < 3; i++) for (int c = 0; c < 3; c++) if (scanf("%lf", &x[i][c]) != 1) return 1;
    for (int i = 0; i < 3; i++) for (int c = 0; c < 3; c++) if (scanf("%lf", &v[i][c]) != 1) return 1;
    if (scanf("%lf", &h) != 1) return 1;
    double Minv, Xc[3], Vc[3], a1[3][3], q2[3], d2[3][3], x5[3][3], v5[3][3], ex[3][3], ev[3][3];
    spl_to_rel<3>(m, x, v, Minv, Xc, Vc);
    spl_acc_rel<3>(k, x, m, a1, q2, d2);
    spl_rkck_step<3, true>(k, x, v, a1, m, Minv, h, x5, v5, ex, ev);
    for (int c = 0; c < 3; c++) Xc[c] = fma(h, Vc[c], Xc[c]);
    double xo[3][3], vo[3][3];
    spl_from_rel<3>(m, x5, v5, Minv, Xc, Vc, xo, vo);
    for (int i = 0; i < 3; i++) for (int c = 0; c < 3; c++) printf("%.17g ", xo[i][c]);
    for (int i = 0; i < 3; i++) for (int c = 0; c < 3; c++) printf("%.17g ", vo[i][c]);
    for (int i = 0; i < 3; i++) for (int c = 0; c < 3; c++) printf("%.17g ", i ? ex[i][c] + ex[0][c] : ex[0][c]);
    for (int i = 0; i < 3; i++) for (int c = 0; c < 3; c++) printf("%.17g ", i ? ev[i][c] + ev[0][c] : ev[0][c]);
    printf("\n");
  }
  return 0;
}
"""


def test_runge_kutta_relative_step_host():
    # the system-per-lane Runge-Kutta kernel's step (star-relative coordinates, Nystrom
    # stages, inertial error vectors rebuilt from the relative ones), compiled as host
    # code, against the oracle's Cash-Karp step in inertial coordinates
    import oracle as O
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    import tempfile
    common = open(COMMON).read()
    herm = open(HERMITE).read()
    rk = open(RK).read()
    f64k = re.search(r"struct F64k \{.*?kadd\(const F64k &k, double a, double b\) \{ return fma\(a, k.one, b\); \}\n",
                     common, re.S).group(0)
    frames = herm[herm.index("// Coordinates relative to body 0"):
                  herm.index("// Acceleration and jerk of bodies k = 1..N-1 relative to body 0")]
    ck = re.search(r"struct CK \{.*?\n\};\n", rk, re.S).group(0)
    ckn = re.search(r"struct CKN \{.*?\n\};\n", rk, re.S).group(0)
    acc = re.search(r"template <int N>\n__device__ __forceinline__ void spl_acc_rel\(.*?\n\}\n", rk, re.S).group(0)
    step = re.search(r"template <int N, bool E>\n__device__ __forceinline__ void spl_rkck_step\(.*?\n\}\n", rk,
                     re.S).group(0)
    prog = ("#include <cmath>\n#include <cstdio>\nusing std::fabs; using std::fma; using std::sqrt; using std::fmax;\n"
            "#define __device__\n#define __forceinline__ inline\n#define __noinline__\n"
            "static inline double rsqrt(double x) { return 1.0 / std::sqrt(x); }\n"
            "namespace swarm {\n" + f64k + frames + ck + ckn + acc + step + "}\n" + RK_MAIN)
    d = tempfile.mkdtemp()
    with open(os.path.join(d, "k.cpp"), "w") as f:
        f.write(prog)
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-Wno-unknown-pragmas", "-o",
                    os.path.join(d, "k"), os.path.join(d, "k.cpp")], check=True)
    rng = np.random.default_rng(11)
    cases, lines = [], []
    for t in range(40):
        m = np.array([1.0, *rng.uniform(1e-5, 1e-3, 2)]) if t % 4 else rng.uniform(0.3, 1.0, 3)
        x = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [-2.2, 0.4, 0.0]]) + 0.05 * rng.standard_normal((3, 3))
        v = np.array([[0.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, -0.65, 0.02]]) + 0.02 * rng.standard_normal((3, 3))
        h = float(rng.uniform(0.05, 0.15))  # error vectors well above the oracle's cancellation noise
        cases.append((m, x, v, h))
        lines.append(" ".join(repr(float(q)) for q in [*m, *x.ravel(), *v.ravel(), h]))
    out = subprocess.run([os.path.join(d, "k")], input="\n".join(lines), capture_output=True, text=True,
                         check=True).stdout.strip().split("\n")
    worst = np.zeros(4)
    for (m, x, v, h), row in zip(cases, out):
        r = np.array(list(map(float, row.split()))).reshape(4, 3, 3)
        xo, vo, _, err = O.rkck_step(m, x, v, h)
        for q, ref in enumerate((xo, vo, err[:3], err[3:])):
            worst[q] = max(worst[q], np.max(np.abs(r[q] - ref)) / np.max(np.abs(ref)))
        assert np.max(np.abs(r[0] - xo)) <= 1e-14 * np.max(np.abs(xo))
        assert np.max(np.abs(r[1] - vo)) <= 1e-14 * np.max(np.abs(vo))
        # the oracle's error vector carries the cancellation of the stage velocities; the
        # kernel's carries none
        assert np.max(np.abs(r[2] - err[:3])) <= 1e-6 * np.max(np.abs(err[:3]))
        assert np.max(np.abs(r[3] - err[3:])) <= 1e-6 * np.max(np.abs(err[3:]))
    print("relative Runge-Kutta step against the oracle:", worst)


MONITOR_MAIN = r"""
using namespace swarm;
int main() {
  // per line: ce mi mj m0 d2 q2i q2j -> close_encounter(d2, hill_kc(...), q2i, q2j)
  const F64k k = {0.0, -1.0, 1.0};
  double ce, mi, mj, m0, d2, qi, qj;
  while (scanf("%lf %lf %lf %lf %lf %lf %lf", &ce, &mi, &mj, &m0, &d2, &qi, &qj) == 7)
    printf("%d\n", close_encounter(k, d2, hill_kc(ce, mi, mj, m0), qi, qj) ? 1 : 0);
  // nonneg_lt against the FP64 order on non-negative values, including 0, subnormals, inf
  const double vals[] = {0.0, 4.9e-324, 2.2e-308, 1e-300, 1e-20, 0.5, 1.0, 1.0000000000000002, 3.0, 1e300,
                         1.7976931348623157e308, INFINITY};
  int bad = 0;
  for (double a : vals) for (double b : vals) bad += nonneg_lt(a, b) != (a < b);
  printf("order %d\n", bad);
  return 0;
}
"""


def test_monitor_host():
    # the monitor's close-encounter test (mutual Hill radius, with its square-root-free
    # shortcut and integer compare) against the definition of the reading, evaluated in
    # 40-digit arithmetic, on cases clustered at the boundary; and the integer order of
    # non-negative doubles
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    import tempfile
    common = open(COMMON).read()
    herm = open(HERMITE).read()
    f64k = re.search(r"struct F64k \{.*?kadd\(const F64k &k, double a, double b\) \{ return fma\(a, k.one, b\); \}\n",
                     common, re.S).group(0)
    lt = re.search(r"__device__ __forceinline__ bool nonneg_lt\(double a, double b\) \{.*?\n\}\n", common,
                   re.S).group(0)
    ce = re.search(r"__device__ __forceinline__ bool close_encounter\(.*?\n\}\n", herm, re.S).group(0)
    kc = re.search(r"__device__ __forceinline__ double hill_kc\(.*?\n\}\n", herm, re.S).group(0)
    prog = ("#include <cmath>\n#include <cstdio>\n#include <cstring>\n"
            "using std::fabs; using std::fma; using std::sqrt; using std::cbrt;\n"
            "#define __device__\n#define __forceinline__ inline\n"
            "static inline long long __double_as_longlong(double x) { long long b; std::memcpy(&b, &x, 8); return b; }\n"
            "namespace swarm {\n" + f64k + lt + ce + kc + "}\n" + MONITOR_MAIN)
    d = tempfile.mkdtemp()
    with open(os.path.join(d, "m.cpp"), "w") as f:
        f.write(prog)
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-o", os.path.join(d, "m"),
                    os.path.join(d, "m.cpp")], check=True)
    rng = np.random.default_rng(3)
    rows, want = [], []
    mp.mp.dps = 40
    for _ in range(3000):
        cef, mi, mj = 3.0, 10 ** rng.uniform(-5, -3), 10 ** rng.uniform(-5, -3)
        qi, qj = rng.uniform(0.5, 5.0, 2)
        rh = float(((mp.mpf(mi) + mj) / 3) ** (mp.mpf(1) / 3) * (mp.mpf(qi) + qj) / 2)
        dist = cef * rh * (1 + float(rng.choice([-1, 1])) * 10 ** rng.uniform(-12, -1))
        if rng.uniform() < 0.1:
            dist = float(rng.uniform(0.0, 10.0))
        d2, q2i, q2j = dist * dist, qi * qi, qj * qj
        rows.append(" ".join(repr(float(t)) for t in [cef, mi, mj, 1.0, d2, q2i, q2j]))
        # the definition on the same (rounded) inputs: |d| < ce R_H, R_H = ((mi+mj)/3)^(1/3) (|Qi|+|Qj|)/2
        R = ((mp.mpf(mi) + mp.mpf(mj)) / 3) ** (mp.mpf(1) / 3) * (mp.sqrt(mp.mpf(q2i)) + mp.sqrt(mp.mpf(q2j))) / 2
        margin = abs(mp.sqrt(mp.mpf(d2)) - cef * R) / (cef * R)
        want.append((mp.sqrt(mp.mpf(d2)) < cef * R, float(margin)))
    out = subprocess.run([os.path.join(d, "m")], input="\n".join(rows), capture_output=True, text=True,
                         check=True).stdout.strip().split("\n")
    assert out[-1] == "order 0"
    got = [s == "1" for s in out[:-1]]
    for g, (w, margin) in zip(got, want):
        # outside a few units of round-off from the boundary the kernel decides as the definition
        if margin > 1e-14:
            assert g == w, margin
    assert sum(got) > 500 and sum(not g for g in got) > 500  # both outcomes exercised


# Plausible mistakes planted in copies of the kernel sources: each must fail one of the
# host checks above (the GPU parity tests are the gate for the kernels; these show that the
# host checks are sharp enough to stand beside them).
KERNEL_MUTANTS = [
    ("nystrom_product_sign", "rkck_impl.cuh", "A62 = -805.0 / 4096.0", "A62 = 805.0 / 4096.0", "constants"),
    ("error_weight", "rkck_impl.cuh", "E5 = 277.0 / 114688.0", "E5 = 277.0 / 114689.0", "constants"),
    ("stumpff_term", "mvs_impl.cuh", "c2 = fma(z, c2, 1.0 / 40320.0);", "c2 = fma(z, c2, 1.0 / 40321.0);", "series"),
    ("stumpff_doubling", "mvs_impl.cuh", "c3 = 0.25 * fma(c0, c3, c2);", "c3 = 0.5 * fma(c0, c3, c2);", "doubling"),
    ("kepler_taylor_sign", "mvs_impl.cuh", "const double U2n = fma(-aU1, d3, fma(U0, d2, fma(U1, d, U2)));",
     "const double U2n = fma(-aU1, d3, fma(U0, d2, fma(-U1, d, U2)));", "kepler"),
    ("kepler_start_sign", "mvs_impl.cuh", "const double T2 = kmul(k, kmul(k, -0.5, Pu), su);",
     "const double T2 = kmul(k, kmul(k, 0.5, Pu), su);", "kepler"),
    ("kepler_fdot_sign", "mvs_impl.cuh", "kmul(k, kmul(k, -K.smu, U1), kmul(k, u, rinv))",
     "kmul(k, kmul(k, K.smu, U1), kmul(k, u, rinv))", "kepler"),
    ("relative_indirect_sign", "hermite.cuh", "A[k][c] = fma(-m0s[k], X[k][c], -IA[c]);",
     "A[k][c] = fma(-m0s[k], X[k][c], IA[c]);", "relative"),
    ("series_refinement_sign", "hermite.cuh", "fma(0.375, del[i][k], -0.5)", "fma(0.375, del[i][k], 0.5)", "relative"),
    ("rk_body0_error_sign", "rkck_impl.cuh", "ex[0][c] = kmul(k, -sx, Minv);", "ex[0][c] = kmul(k, sx, Minv);",
     "runge_kutta"),
    ("rk_indirect_sign", "rkck_impl.cuh", "A[k][c] = fma(-m0s[k], X[k][c], -A[0][c]);",
     "A[k][c] = fma(-m0s[k], X[k][c], A[0][c]);", "runge_kutta"),
    ("hill_factor", "hermite.cuh", "double k = cbrt((mi + mj) / (3.0 * m0));", "double k = cbrt((mi + mj) / (2.0 * m0));",
     "monitor"),
    ("encounter_shortcut", "hermite.cuh", "kmul(k, kmul(k, 2.0, kc), t)", "kmul(k, kmul(k, 1.0, kc), t)", "monitor"),
]


@pytest.mark.parametrize("name,fname,old,new,check", KERNEL_MUTANTS, ids=[m[0] for m in KERNEL_MUTANTS])
def test_host_checks_catch_planted_kernel_mistakes(name, fname, old, new, check, tmp_path, monkeypatch):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    import test_rkck_constants as rc
    csrc = os.path.dirname(SRC)
    for f in ("common.cuh", "hermite.cuh", "mvs_impl.cuh", "rkck_impl.cuh"):
        text = open(os.path.join(csrc, f)).read()
        if f == fname:
            assert old in text, (name, "the planted text is not in the source")
            text = text.replace(old, new, 1)
        (tmp_path / f).write_text(text)
    here = __import__(__name__)
    monkeypatch.setattr(here, "SRC", str(tmp_path / "mvs_impl.cuh"))
    monkeypatch.setattr(here, "RK", str(tmp_path / "rkck_impl.cuh"))
    monkeypatch.setattr(here, "COMMON", str(tmp_path / "common.cuh"))
    monkeypatch.setattr(here, "HERMITE", str(tmp_path / "hermite.cuh"))
    monkeypatch.setattr(rc, "SRC", str(tmp_path / "rkck_impl.cuh"))
    with pytest.raises(AssertionError):
        if check == "constants":
            rc.test_stage_weights_and_errors_match_the_tableau()
            rc.test_nystrom_products_match_the_tableau()
        elif check == "series":
            check_series_range(build_stumpff(str(tmp_path)))
        elif check == "doubling":
            check_quartering_and_doubling(build_stumpff(str(tmp_path)))
        elif check == "kepler":
            exe = build_kepler(str(tmp_path))
            for e in (0.05, 0.3):
                check_kepler_elliptic(exe, e)
        elif check == "relative":
            test_star_relative_evaluation_host()
        elif check == "runge_kutta":
            test_runge_kutta_relative_step_host()
        elif check == "monitor":
            test_monitor_host()


COEF_MAIN = r"""
using namespace swarm;
int main() {
  double h;
  const F64k k = {0.0, -1.0, 1.0};
  while (scanf("%lf", &h) == 1) {
    HCoef c = hcoef(h), d = hcoef(k, h);
    PCoef p = pcoef(h);
    printf("%.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g\n", c.h, c.h2_2, c.h3_6,
           c.hh, c.h2_12, d.h2_2, d.h3_6, d.hh, d.h2_12, p.pa, p.pj, p.ca, p.cj);
  }
  return 0;
}
"""


def test_step_coefficients_host():
    # the Hermite step's coefficients (Eq. 3 predictor h, h^2/2, h^3/6; the time-symmetric
    # corrector's h/2, h^2/12; the printed Eq. 4 form with 3/20: -3h^2/20, -7h^3/60, 3h^2/20,
    # -h^3/30), both the plain and the DFMA-form builders, against exact fractions
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    import tempfile
    from fractions import Fraction as Fr
    common = open(COMMON).read()
    herm = open(HERMITE).read()
    f64k = re.search(r"struct F64k \{.*?kadd\(const F64k &k, double a, double b\) \{ return fma\(a, k.one, b\); \}\n",
                     common, re.S).group(0)
    coef = herm[herm.index("// Coefficients of one step of length h."):herm.index("__device__ __forceinline__ HCoef hsel(")]
    prog = ("#include <cmath>\n#include <cstdio>\nusing std::fma;\n#define __device__\n#define __forceinline__ inline\n"
            "namespace swarm {\n" + f64k + coef + "}\n" + COEF_MAIN)
    d = tempfile.mkdtemp()
    with open(os.path.join(d, "c.cpp"), "w") as f:
        f.write(prog)
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-o", os.path.join(d, "c"),
                    os.path.join(d, "c.cpp")], check=True)
    hs = [2 * np.pi * 1e-3, -2 * np.pi * 1e-3, 0.05, 1e-7, 3.0]
    out = subprocess.run([os.path.join(d, "c")], input="\n".join(repr(h) for h in hs), capture_output=True, text=True,
                         check=True).stdout.strip().split("\n")
    for h, row in zip(hs, out):
        v = [float(t) for t in row.split()]
        H = Fr(h)
        want = [H, H * H / 2, H ** 3 / 6, H / 2, H * H / 12, H * H / 2, H ** 3 / 6, H / 2, H * H / 12,
                -Fr(3, 20) * H * H, -Fr(7, 60) * H ** 3, Fr(3, 20) * H * H, -Fr(1, 30) * H ** 3]
        for got, w in zip(v, want):
            assert abs(Fr(got) - w) <= abs(w) * Fr(4, 2 ** 53), (h, got, float(w))
