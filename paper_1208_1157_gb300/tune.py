"""Measure the autotuner's mapping choices for the standard workload shapes on this GPU
and save them (swarm_tuner_save) so that later runs load them instead of measuring.

    python -m paper_1208_1157_gb300.tune [output path]

Shapes: the 1024- and 131072-system three-body ensembles, the per-n bins of the
65536-system ragged ensemble (about 5041 systems each), the 16384 x 8 MVS ensemble and
the serving pools (16384 slots per integrator and n)."""
from __future__ import annotations

import os
import sys

from . import swarm as S

DEFAULT_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_gb300.txt")


def shapes():
    out = [(3, S.HERMITE4, 1024), (3, S.HERMITE4, 131072), (8, S.MVS_JACOBI, 16384), (8, S.MVS_DH, 16384)]
    for n in range(3, 16):
        out.append((n, S.HERMITE4, 5041))
        out.append((n, S.HERMITE4, 16384))
        out.append((n, S.MVS_DH, 16384))
    return out


def main(path: str = DEFAULT_PATH) -> None:
    S.tuner_load(path)
    for n, integ, nsys in shapes():
        m, c = S.tuner_choice(n, integ, nsys)
        print(f"n={n:2d} integrator={integ} n_sys={nsys:6d}: mapping {m} ctas/SM {c}", flush=True)
    S.tuner_save(path)
    print("saved", path)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else DEFAULT_PATH)
