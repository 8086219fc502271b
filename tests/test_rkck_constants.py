"""The Cash-Karp constants compiled into the GPU kernels (csrc/rkck_impl.cuh, read as
text: no GPU needed) against the oracle's tableau (Cash & Karp 1990): the stage
coefficients, the 5th-order weights, the error weights, and the composite products of the
Nystrom form (Abar = A A, Bbar = b5 A, Ebar = (b5 - b4) A, c = row sums of A)."""
import os
import re
from fractions import Fraction

import numpy as np

import oracle as O

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1208_1157_gb300", "csrc",
                   "rkck_impl.cuh")


def struct_constants(name):
    """{identifier: exact value} of the `static constexpr double` members of struct `name`."""
    text = open(SRC).read()
    body = re.search(r"struct %s \{(.*?)\n\};" % name, text, re.S).group(1)
    out = {}
    for decl in re.findall(r"static constexpr double (.*?);", body, re.S):
        for item in re.split(r",\s*(?=[A-Z]\w*\s*=)", decl):
            key, expr = item.split("=", 1)
            expr = re.sub(r"(\d+\.\d+)", r"Fraction('\1')", expr)
            out[key.strip()] = eval(expr, {"Fraction": Fraction})
    return out


def exact_tableau():
    c, a, b5, b4 = O.rkck_tableau()
    fr = lambda x: Fraction(float(x)).limit_denominator(10 ** 7)
    A = [[fr(a[i][j]) for j in range(6)] for i in range(6)]
    return [fr(x) for x in c], A, [fr(x) for x in b5], [fr(x) for x in b4]


def test_stage_weights_and_errors_match_the_tableau():
    c, A, b5, b4 = exact_tableau()
    ck = struct_constants("CK")
    for i in range(2, 7):
        for j in range(1, i):
            assert ck[f"A{i}{j}"] == A[i - 1][j - 1], (i, j)
    for j in (1, 3, 4, 6):
        assert ck[f"B{j}"] == b5[j - 1]
    assert b5[1] == 0 and b5[4] == 0
    for j in (1, 3, 4, 5, 6):
        assert ck[f"E{j}"] == b5[j - 1] - b4[j - 1]
    assert b4[1] == 0


def test_nystrom_products_match_the_tableau():
    c, A, b5, b4 = exact_tableau()
    ckn = struct_constants("CKN")
    Ab = [[sum(A[i][k] * A[k][l] for k in range(6)) for l in range(6)] for i in range(6)]
    Bb = [sum(b5[k] * A[k][l] for k in range(6)) for l in range(6)]
    Eb = [sum((b5[k] - b4[k]) * A[k][l] for k in range(6)) for l in range(6)]
    for i in (2, 3, 4, 6):
        assert ckn[f"C{i}"] == c[i - 1] == sum(A[i - 1])
    assert c[4] == 1  # stage 5 sits at the end of the step
    used = {3: (1,), 4: (1, 2), 5: (1, 2, 3), 6: (1, 2, 3, 4)}
    for i, ls in used.items():
        for l in range(1, 7):
            if l in ls:
                assert ckn[f"A{i}{l}"] == Ab[i - 1][l - 1], (i, l)
            else:
                assert Ab[i - 1][l - 1] == 0, (i, l)  # terms the kernel omits vanish
    for l in range(1, 7):
        if l in (1, 3, 4, 5):
            assert ckn[f"B{l}"] == Bb[l - 1]
            assert ckn[f"E{l}"] == Eb[l - 1]
        else:
            assert Bb[l - 1] == 0 and Eb[l - 1] == 0
    # the error weights sum to zero, which the Nystrom error form relies on
    assert sum(b5) == 1 and sum(b4) == 1


def test_nystrom_step_equals_the_stage_velocity_step():
    # one Cash-Karp step of a 3-body system in the Nystrom form of the constants above
    # against the oracle's step (stage velocities): same 5th-order solution to round-off
    ckn = {k: float(v) for k, v in struct_constants("CKN").items()}
    ck = {k: float(v) for k, v in struct_constants("CK").items()}
    m = np.array([1.0, 1e-3, 2e-3])
    x = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [-0.3, 1.9, 0.05]])
    v = np.array([[0.0, 0.0, 0.0], [-0.05, 1.0, 0.0], [-0.7, -0.1, 0.01]])
    h = 0.05

    def acc(p):
        a = np.zeros_like(p)
        for i in range(3):
            for j in range(3):
                if i != j:
                    d = p[j] - p[i]
                    a[i] += m[j] * d / np.linalg.norm(d) ** 3
        return a

    a1 = acc(x)
    a2 = acc(x + ckn["C2"] * h * v)
    a3 = acc(x + ckn["C3"] * h * v + h * h * ckn["A31"] * a1)
    a4 = acc(x + ckn["C4"] * h * v + h * h * (ckn["A41"] * a1 + ckn["A42"] * a2))
    a5 = acc(x + h * v + h * h * (ckn["A51"] * a1 + ckn["A52"] * a2 + ckn["A53"] * a3))
    a6 = acc(x + ckn["C6"] * h * v + h * h * (ckn["A61"] * a1 + ckn["A62"] * a2 + ckn["A63"] * a3 + ckn["A64"] * a4))
    x5 = x + h * v + h * h * (ckn["B1"] * a1 + ckn["B3"] * a3 + ckn["B4"] * a4 + ckn["B5"] * a5)
    v5 = v + h * (ck["B1"] * a1 + ck["B3"] * a3 + ck["B4"] * a4 + ck["B6"] * a6)
    ex = h * h * (ckn["E1"] * a1 + ckn["E3"] * a3 + ckn["E4"] * a4 + ckn["E5"] * a5)
    xo, vo, _, err = O.rkck_step(m, x, v, h)
    assert np.max(np.abs(x5 - xo)) <= 1e-15 * np.max(np.abs(xo))
    assert np.max(np.abs(v5 - vo)) <= 1e-15 * np.max(np.abs(vo))
    # the oracle forms the position error with the stage velocities' cancellation
    assert np.max(np.abs(ex - err[:3])) <= 1e-6 * np.max(np.abs(err[:3]))
