"""Plant plausible mistakes in the oracle's C source and check that the pins catch each.

Every mutant is compiled from a modified copy of oracle.c (on the CPU) and the pin
suite is run against it in a subprocess; a mutant that passes every pin would mean
the pins cannot see that kind of slip.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "jerk_sign": ("ji[c] += m[j] * (u[c] - s * r[c]) * rinv3;", "ji[c] += m[j] * (u[c] + s * r[c]) * rinv3;"),
    "jerk_factor3": ("double s = 3.0 * rv / r2;", "double s = rv / r2;"),
    "star_not_last": ("for (int j = n - 1; j >= 0; j--) {\n      if (j == i) continue;\n      double r[3], u[3];",
                      "for (int j = 0; j < n; j++) {\n      if (j == i) continue;\n      double r[3], u[3];"),
    "predictor_no_jerk": ("xp[q] = x0[q] + v0[q] * dt + a0[q] * dt2 / 2.0 + j0[q] * dt3 / 6.0;",
                          "xp[q] = x0[q] + v0[q] * dt + a0[q] * dt2 / 2.0;"),
    "printed_3_10": ("xk[q] = xp[q] - 3.0 / 20.0 *", "xk[q] = xp[q] - 3.0 / 10.0 *"),
    "corrector_sign": ("xk[q] = x0[q] + (v0[q] + vk[q]) * dt / 2.0 + (a0[q] - ak[q]) * dt2 / 12.0;",
                       "xk[q] = x0[q] + (v0[q] + vk[q]) * dt / 2.0 + (ak[q] - a0[q]) * dt2 / 12.0;"),
    "energy_double_count": ("for (int j = i + 1; j < n; j++) {\n      double r[3];\n      for (int c = 0; c < 3; c++) r[c] = x[3 * j + c] - xi[c];",
                            "for (int j = 0; j < n; j++) {\n      if (j == i) continue;\n      double r[3];\n      for (int c = 0; c < 3; c++) r[c] = x[3 * j + c] - xi[c];"),
    "stumpff_series_sign": ("t2 *= -z / ((2.0 * k + 3.0) * (2.0 * k + 4.0));", "t2 *= z / ((2.0 * k + 3.0) * (2.0 * k + 4.0));"),
    "kepler_fdot": ("double fd = smu / (rnorm * r0) * chi * (z * S - 1.0);", "double fd = smu / (rnorm * r0) * chi * (z * S + 1.0);"),
    "dh_kick_with_star": ("for (int j = n - 1; j >= 1; j--) {\n      if (j == i) continue;\n      double r[3];\n      for (int c = 0; c < 3; c++) r[c] = q[3 * j + c] - q[3 * i + c];",
                          "for (int j = n - 1; j >= 0; j--) {\n      if (j == i) continue;\n      double r[3];\n      for (int c = 0; c < 3; c++) r[c] = (j ? q[3 * j + c] : 0.0) - q[3 * i + c];"),
    "dh_drift_mass": ("q[3 * i + c] += h * p[c] / m[0];", "q[3 * i + c] += h * p[c];"),
    "jacobi_mu": ("double mu = m[0] * eta_i / eta;", "double mu = m[0];"),
    "jacobi_transform": ("R[c] -= m[i] / eta[i] * r[3 * i + c];", "R[c] -= m[i] / eta[i - 1] * r[3 * i + c];"),
    "adaptive_dt_square": ("s += dot3(j, j) / dot3(a, a);", "s += sqrt(dot3(j, j) / dot3(a, a));"),
    "monitor_hill_cube": ("cbrt((m[i] + m[j]) / (3.0 * m[0]))", "sqrt((m[i] + m[j]) / (3.0 * m[0]))"),
    "rkck_b5_typo": ("125.0 / 594.0", "125.0 / 549.0"),
    "rkck_propagate_b4": ("sx += RK_B5[s] * kx[s][q];", "sx += RK_B4[s] * kx[s][q];"),
    "rkck_stage_velocity": ("for (int q = 0; q < d; q++) kx[s][q] = vs[q];", "for (int q = 0; q < d; q++) kx[s][q] = v[q];"),
    "rkck_accept_loose": ("if (err <= 1.0) {", "if (err <= 100.0) {"),
    "rv_wrong_body": ("rv[k] = v[0] * los[0] + v[1] * los[1] + v[2] * los[2];",
                      "rv[k] = v[3] * los[0] + v[4] * los[1] + v[5] * los[2];"),
    "rkck_error_weights": ("tx += (RK_B5[s] - RK_B4[s]) * kx[s][q];", "tx += (RK_B5[s] - RK_B4[s]) * kv[s][q];"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mut = tmp_path / "oracle.c"
    mut.write_text(src.replace(old, new))
    (tmp_path / "oracle.h").write_text(open(os.path.join(ROOT, "oracle", "oracle.h")).read())
    so = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so), str(mut), "-lm"])
    env = dict(os.environ, ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"
