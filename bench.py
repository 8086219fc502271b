#!/usr/bin/env python
"""Benchmark of the FP64 ensemble integrator on GB300.

One bench step = one swarm_integrate call advancing the paper-shaped ensemble
(131072 systems x 3 bodies, Hermite-4 P(EC)^2, dt = 1e-3 inner periods) by 10^4 steps
with energy/angular-momentum logging every 1000 steps and the close-encounter /
ejection monitor on.  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank integrates its own independent ensemble (weak scaling, no
collective on the data path; the barrier and the max over ranks are for timing only).
--impl reference times the CPU oracle (plain single-threaded C, one process per host
core) on a bounded sample of the same workload.
"""
import argparse
import glob
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

TWO_PI = 2.0 * math.pi
DT = TWO_PI * 1e-3
N_SYS = 131072
N_BODY = 3
STEPS_PER_CALL = 10000
LOG_EVERY = 1000
METRIC = "FP64 system-steps/s & pair-interactions/s vs FP64 peak; serving p50/p99 latency"
WORKLOAD = "paper-shaped ensemble: 131072 systems x 3 bodies (seed 2), Hermite-4 P(EC)^2 FP64, 10^4 steps per call, dt = 2pi 1e-3, E/L logged every 1000 steps, stops on (3 Hill radii, 100 AU)"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ------------------------------------------------------------------ operation counts
def hermite_flops_per_system_step(n, n_corr=2):
    """FP64 operations of the implemented Hermite step, system per lane (a DFMA counts 2,
    rsqrt 1).  The step runs on coordinates relative to body 0 plus the barycentre.

    per evaluation (n_corr + 1 per step):
      each body k >= 1 with body 0: |X|^2, X.V (2 x 5), rsqrt (1), rho^2, rho^3 (2),
        -3 (X.V) rho^2 (2), m_k s, m_0 s (2), w = V + c X (6), the bases of A_k and J_k
        (2 x 3 DFMA = 12): 35;
      the sums m_j s_j X_j and m_j s_j w_j over k >= 1: 6 + 12 (n - 2);
      each pair of bodies i, k >= 1: 6 differences, 2 dot products (10), rsqrt (1),
        rho^2, rho^3 (2), -3 (r.u) rho^2 (2), w (6), each body's share (1 + 12, twice) = 53;
    per component of bodies k >= 1 and step: predictor 5 DFMA, corrector bases 4 DFMA,
      4 DFMA per corrector pass: (9 + 4 n_corr) * 2; the barycentre's drift 3 DFMA = 6."""
    P = (n - 1) * (n - 2) // 2
    per_eval = 35 * (n - 1) + 6 + 12 * (n - 2) + 53 * P
    return (n_corr + 1) * per_eval + 3 * (n - 1) * (9 + 4 * n_corr) * 2 + 6


def scope_hermite_flops(n, n_corr=2):
    """The scope table's count of the Hermite step (row a2-a4): ~58 flops per unique pair
    and evaluation (differences 6, r^2 5, r.u 5, rsqrt 1, rho^2 and rho^3 2, the jerk factor
    2, each body's share 19), n_corr + 1 evaluations, and 34 flops per body component for
    the predictor and the correctors: 3 P 58 + 3 n 34 at n_corr = 2 (n = 3: 828)."""
    P = n * (n - 1) // 2
    return (n_corr + 1) * P * 58 + 3 * n * 34


def scope_mvs_flops(n, newton=1.0, jacobi=True):
    """The scope table's count of the MVS step (rows a7-a9): ~25 flops per planet pair of
    the kick (Jacobi: every pair, the star's included, as implemented), per planet ~40 flops
    of Kepler set-up, ~30 per Newton iteration (measured count) and ~30 for f, g, and ~6n
    for the drifts."""
    pairs = n * (n - 1) // 2 if jacobi else (n - 1) * (n - 2) // 2
    return 25 * pairs + (n - 1) * (40 + 30 * newton + 30) + 6 * n


def rkck_flops(n):
    """Implemented Runge-Kutta Cash-Karp step (six acceleration evaluations, Nystrom
    stages): system per lane in star-relative coordinates for n <= 3,
    6 [16 (n-1) + 3 + 6 (n-2) + 25 P'] + 3 (n-1) 54 + 11; body per lane above,
    6 P 25 + 3 n 54 + 5 n (P = n (n-1)/2, P' = (n-1)(n-2)/2)."""
    if n <= 3:
        Pp = (n - 1) * (n - 2) // 2
        return 6 * (16 * (n - 1) + 3 + 6 * (n - 2) + 25 * Pp) + 3 * (n - 1) * 54 + 11
    return 6 * (n * (n - 1) // 2) * 25 + 3 * n * 54 + 5 * n


def steps_by_system(ens, out, dt, t0=0.0):
    """Steps each system took in a fixed-step call (its final time against its start)."""
    import numpy as np

    return np.round(np.abs(np.asarray(out["time"]) - t0) / abs(dt)).astype(np.int64)


def source_hash(patterns):
    h = hashlib.sha256()
    for p in sorted(sum((glob.glob(os.path.join(ROOT, q)) for q in patterns), [])):
        h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


# the sources of the benchmark's kernel (hermite_uniform_kernel, system per lane)
HERMITE_SOURCES = ["paper_1208_1157_gb300/csrc/hermite.cuh", "paper_1208_1157_gb300/csrc/hermite_impl.cuh",
                   "paper_1208_1157_gb300/csrc/hermite_uniform_spl.cu", "paper_1208_1157_gb300/csrc/common.cuh"]


def traffic_per_launch(kernel, systems):
    """DRAM bytes per launch from the committed ncu summary, scaled to `systems`, or None
    when the kernel sources changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path)).get(kernel)
        if not d or d.get("source_hash") != source_hash(HERMITE_SOURCES):
            return None
        return d["dram_bytes_per_system"] * systems
    except Exception:
        return None


# ------------------------------------------------------------------ clocks
class Clocks:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception as ex:  # no nvidia-smi: report unknown clocks
            log("clock sampling unavailable:", ex)
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        rows = []
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), float(f[3]), f[5:9]))
            except ValueError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        loaded = [r for r in rows if r[2] > 250.0] or rows
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


# ------------------------------------------------------------------ CPU oracle leg
def _oracle_chunk(args):
    seed, idx, steps = args
    sys.path.insert(0, ROOT)
    import oracle as O
    from paper_1208_1157_gb300 import ics

    ens = ics.subset(ics.three_body(int(max(idx)) + 1, seed), idx)
    t = time.perf_counter()
    O.integrate(ens, steps * DT, DT, O.HERMITE, ce_factor=3.0, eject_radius=100.0)
    return time.perf_counter() - t


def _oracle_config_rate(name):
    """Single-core oracle rate on a small sample of one workload (system-steps/s)."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import oracle as O
    from paper_1208_1157_gb300 import ics

    if name == "c1_three_body_1024":
        ens, integ, dt, steps = ics.three_body(1024, 1), O.HERMITE, DT, 1000
    elif name == "c2_three_body_sample_512":
        ens, integ, dt, steps = ics.subset(ics.three_body(512 * 64, 2), list(range(0, 512 * 64, 64))), O.HERMITE, DT, 2000
    elif name == "c3_ragged_sample_1024":
        ens, integ, dt, steps = ics.subset(ics.ragged(1024 * 64, 3), list(range(0, 1024 * 64, 64))), O.HERMITE, DT, 100
    else:  # c4 compact 8-body sample, Jacobi MVS
        ens, integ, dt, steps = ics.subset(ics.mvs_compact(256 * 64, 4), list(range(0, 256 * 64, 64))), O.MVS_JACOBI, TWO_PI / 20, 2000
    t = time.perf_counter()
    out = O.integrate(ens, steps * dt, dt, integ, ce_factor=3.0, eject_radius=100.0)
    wall = time.perf_counter() - t
    done = float(np.sum(np.round(out["time"] / dt)))
    return name, {"system_steps_per_s": done / wall, "systems": len(ens["n_body"]), "steps_per_system": steps,
                  "wall_s": wall}


def oracle_config_rates():
    """The oracle on one host core per workload (spawned before any CUDA use): C1 whole,
    every 64th system of C2, C3 and C4."""
    ctx = mp.get_context("spawn")
    names = ["c1_three_body_1024", "c2_three_body_sample_512", "c3_ragged_sample_1024", "c4_mvs_jacobi_sample_256"]
    with ctx.Pool(len(names)) as pool:
        return dict(pool.map(_oracle_config_rate, names))


def oracle_throughput(target_s=15.0, steps=STEPS_PER_CALL, seed=2):
    """The oracle as it stands, one process per host core (spawned before any CUDA use),
    on a sample of systems sized for about target_s seconds of wall time."""
    import oracle as O

    O.build()
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        # calibrate: one system for 1000 steps on one core
        t1 = pool.map(_oracle_chunk, [(seed, [0], 1000)])[0]
        per_sys = t1 * steps / 1000.0
        per_core = max(1, int(target_s / max(per_sys, 1e-6)))
        S = min(cores * per_core, N_SYS)
        chunks = [(seed, list(range(c, S, cores)), steps) for c in range(cores) if c < S]
        t = time.perf_counter()
        pool.map(_oracle_chunk, chunks)
        wall = time.perf_counter() - t
    return {"value": S * steps / wall, "unit": "system-steps/s", "cores": min(cores, S), "kind": "oracle",
            "sample": f"{S} of the {N_SYS} systems (seed 2), {steps} Hermite steps each, one process per core",
            "wall_s": wall, "build": "gcc " + " ".join(O.CFLAGS)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_step = []
    res = None
    for k in range(args.warmup + args.steps):
        res = oracle_throughput(target_s=args.ref_seconds)
        if k >= args.warmup:
            per_step.append(res)
    value = statistics.median(r["value"] for r in per_step)
    cpu = dict(per_step[-1])
    cpu["value"] = value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "system-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * statistics.median(r["wall_s"] for r in per_step),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": cpu["sample"]},
            "cpu_baseline": cpu, "e2e": {"value": value, "unit": "system-steps/s", "h2d_bytes_per_step": 0,
                                          "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ranks
def rank_seed(rank):
    """Each rank integrates its own independent ensemble (no exchange between ranks)."""
    return 2 + 1000 * rank


def reduce_over_ranks(dist, maxv, sumv, device):
    """(max over ranks of each of maxv, sum over ranks of each of sumv): the timing
    reduction of the weak-scaling benchmark; no data-path collective exists."""
    import torch

    t = torch.tensor(list(maxv) + list(sumv), dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    k = len(maxv)
    return [float(v) for v in mx[:k]], [float(v) for v in sm[k:]]


# ------------------------------------------------------------------ our path
def secondary(S, torch, stream, peak):
    """Short measurements of the other rows of the hot path (not the headline value).
    Every entry carries its FP64 work as counted by the scope table (Hermite, MVS) or by
    the implemented formula (Runge-Kutta), summed over the steps each system took, and that
    work per kernel second as a fraction of the measured FP64 peak."""
    import numpy as np

    from paper_1208_1157_gb300 import ics

    out = {}

    def account(o, flops, sec, how):
        o["fp64_flops"] = float(flops)
        o["fp64_tflops"] = flops / sec / 1e12
        o["fp64_frac"] = flops / sec / peak
        o["fp64_count"] = how

    def timed(ens, t_end, integ, dt, mapping=0, ce=3.0, ej=100.0, ctas=0, outcome=False):
        with S.Ensemble(ens, stream=stream) as e:
            e.set_option(S.OPT_MAPPING, mapping)
            e.set_option(S.OPT_CTAS_PER_SM, ctas)
            e.set_stop(ce, ej)
            e.integrate(min(t_end, 2 * dt), integ, dt)  # warm-up (tuner, caches)
            e.set_state(ens["pos"], ens["vel"], time=[0.0] * len(ens["n_body"]),
                        status=[0] * len(ens["n_body"]))
            E0 = e.diagnostics()[0] if outcome else None
            e.integrate(t_end, integ, dt)
            st = e.stats()
            state = e.state()
            if outcome:
                E1 = e.diagnostics()[0]
        status = state["status"]
        sec = st["kernel_ms"] * 1e-3
        o = {"system_steps_per_s": st["system_steps"] / sec, "pair_interactions_per_s": st["pair_evaluations"] / sec,
             "kernel_ms": st["kernel_ms"], "launches": st["kernel_launches"], "system_steps": st["system_steps"],
             "kepler_iterations": st["kepler_iterations"]}
        nb = np.asarray(ens["n_body"])
        if integ in (S.HERMITE4, S.MVS_DH, S.MVS_JACOBI, S.RKCK):
            steps = steps_by_system(ens, state, dt)
        else:  # adaptive: the counters' total, all systems alike
            steps = np.full(len(nb), st["system_steps"] / len(nb))
        if integ in (S.HERMITE4, S.HERMITE4_ADAPTIVE):
            extra = 8 * nb if integ == S.HERMITE4_ADAPTIVE else 0  # the Eq. 5 sum
            flops = np.sum((np.vectorize(scope_hermite_flops)(nb) + extra) * steps)
            account(o, flops, sec, "scope table: 3 P 58 + 3 n 34 per Hermite step" +
                    (" + 8 n for Eq. 5" if integ == S.HERMITE4_ADAPTIVE else ""))
        elif integ in (S.MVS_DH, S.MVS_JACOBI):
            newton = st["kepler_iterations"] / max(1.0, float(np.sum(steps * (nb - 1))))
            jac = integ == S.MVS_JACOBI
            flops = np.sum(np.vectorize(lambda n: scope_mvs_flops(n, newton, jac))(nb) * steps)
            account(o, flops, sec, "scope table: 25 per kicked pair + (n-1)(40 + 30 I + 30) + 6 n per MVS step, "
                    f"I = {newton:.4f} measured Newton iterations per drift")
            o["newton_iterations_per_drift"] = newton
        else:
            flops = np.sum(np.vectorize(rkck_flops)(nb) * steps)
            account(o, flops, sec, "implemented Cash-Karp step (six evaluations, Nystrom stages)")
        if outcome:
            # stop outcomes, |dE/E| of the systems that reached t_end
            names = ["active", "done", "close_encounter", "ejected", "kepler_noconv", "nonfinite", "span_limit"]
            cnt = np.bincount(status, minlength=len(names))
            dE = np.abs(E1 / E0 - 1.0)[status == 1]
            o["status_counts"] = {names[k]: int(cnt[k]) for k in range(len(names))}
            if len(dE):
                o["energy_error_done"] = {"p50": float(np.percentile(dE, 50)), "p90": float(np.percentile(dE, 90)),
                                          "max": float(dE.max())}
        return o

    c2 = ics.three_body(N_SYS, seed=2)
    out["c2_plain_one_launch_per_step_500"] = timed(c2, 500 * DT, S.HERMITE4, DT, mapping=S.MAP_PLAIN_PER_STEP)
    c1 = ics.three_body(1024, seed=1)
    out["c1_plain_one_launch_per_step_1000"] = timed(c1, 1000 * DT, S.HERMITE4, DT, mapping=S.MAP_PLAIN_PER_STEP)
    out["c1_persistent_1000"] = timed(c1, 1000 * DT, S.HERMITE4, DT)
    out["c2_persistent_500"] = timed(c2, 500 * DT, S.HERMITE4, DT)
    out["c2_persistent_body_per_lane_500"] = timed(c2, 500 * DT, S.HERMITE4, DT, mapping=S.MAP_BODY_PER_LANE)
    out["c2_persistent_system_per_lane_500"] = timed(c2, 500 * DT, S.HERMITE4, DT, mapping=S.MAP_SYSTEM_PER_LANE)
    out["c2_persistent_system_per_lane_1cta_500"] = timed(c2, 500 * DT, S.HERMITE4, DT, mapping=S.MAP_SYSTEM_PER_LANE,
                                                          ctas=1)
    out["c2_persistent_body_per_lane_1cta_500"] = timed(c2, 500 * DT, S.HERMITE4, DT, mapping=S.MAP_BODY_PER_LANE,
                                                        ctas=1)
    out["c2_persistent_system_per_lane_3cta_500"] = timed(c2, 500 * DT, S.HERMITE4, DT, mapping=S.MAP_SYSTEM_PER_LANE,
                                                          ctas=3)
    c3 = ics.ragged(65536, seed=3)
    out["c3_ragged_hermite_per_bin_launches_1e4_steps"] = timed_per_bin(S, stream, c3, 1e4 * DT, DT, peak)
    out["c3_ragged_hermite_single_launch_1e4_steps"] = timed_per_bin(S, stream, c3, 1e4 * DT, DT, peak, single=1)
    out["c3_ragged_hermite_bins_alone_500_steps"] = bins_alone(S, stream, c3, 500, DT, peak)
    c4 = ics.mvs_compact(16384, seed=4)
    out["c4_mvs_jacobi_2000_steps"] = timed(c4, 2000 * TWO_PI / 20, S.MVS_JACOBI, TWO_PI / 20)
    out["c4_mvs_jacobi_2000_steps_2cta"] = timed(c4, 2000 * TWO_PI / 20, S.MVS_JACOBI, TWO_PI / 20, ctas=2)
    out["c4_mvs_jacobi_1e5_steps"] = timed(c4, 1e5 * TWO_PI / 20, S.MVS_JACOBI, TWO_PI / 20, outcome=True)
    out["c4_mvs_jacobi_1e5_steps_2cta"] = timed(c4, 1e5 * TWO_PI / 20, S.MVS_JACOBI, TWO_PI / 20, ctas=2)
    out["c4_mvs_dh_1e5_steps"] = timed(c4, 1e5 * TWO_PI / 20, S.MVS_DH, TWO_PI / 20, outcome=True)
    out["c2_hermite_adaptive_tau_0.01_one_period"] = timed(c2, TWO_PI, S.HERMITE4_ADAPTIVE, 0.01)
    out["c2_hermite_adaptive_tau_0.01_one_period_2cta"] = timed(c2, TWO_PI, S.HERMITE4_ADAPTIVE, 0.01, ctas=2)
    out["c2_rkck_fixed_500"] = timed(c2, 500 * DT, S.RKCK, DT)
    out["c2_rkck_fixed_1cta_500"] = timed(c2, 500 * DT, S.RKCK, DT, ctas=1)
    out["c2_rkck_adaptive_eps_1e-12_one_period"] = timed(c2, TWO_PI, S.RKCK_ADAPTIVE, 0.05)
    out["c3_ragged_rkck_100_steps"] = timed(c3, 100 * DT, S.RKCK, DT)
    # the ragged batch against the plain one-launch-per-step kernel on the same systems
    # (the plain kernel has n <= 8): 65536 systems, n = 3..8, 500 steps
    c3s = ics.ragged(65536, seed=3, n_max=8)
    out["c3_ragged_n3_8_plain_one_launch_per_step_500"] = timed(c3s, 500 * DT, S.HERMITE4, DT,
                                                               mapping=S.MAP_PLAIN_PER_STEP)
    out["c3_ragged_n3_8_persistent_500"] = timed(c3s, 500 * DT, S.HERMITE4, DT)
    c6 = ics.ragged_wide(16384, seed=6)
    out["wide_16_to_32_bodies_hermite_20_steps"] = timed(c6, 20 * DT, S.HERMITE4, DT)
    out["wide_16_to_32_bodies_mvs_jacobi_100_steps"] = timed(c6, 100 * TWO_PI / 20, S.MVS_JACOBI, TWO_PI / 20)
    out["wide_16_to_32_bodies_rkck_20_steps"] = timed(c6, 20 * DT, S.RKCK, DT)
    out["serving"] = serving(S, stream, peak)
    out["serving_vs_plain_hermite_n3_8_t_end_divided_by_1000"] = serving_vs_plain(S, stream, peak)
    out["serving_by_integrator_t_end_divided_by_1000"] = serving_by_integrator(S, stream, peak)
    return out


def timed_per_bin(S, stream, ens, t_end, dt, peak, single=0):
    """The ragged ensemble with one single-bin launch per body count (single = 0, the
    default) or one shared launch over all bins (single = 1); FP64 work by the scope
    table's Hermite count, per body count as well."""
    import numpy as np

    with S.Ensemble(ens, stream=stream) as e:
        e.set_option(S.OPT_SINGLE_LAUNCH, single)
        e.integrate(2 * dt, S.HERMITE4, dt)
        e.set_state(ens["pos"], ens["vel"], time=[0.0] * len(ens["n_body"]), status=[0] * len(ens["n_body"]))
        e.integrate(t_end, S.HERMITE4, dt)
        st = e.stats()
        state = e.state()
    sec = st["kernel_ms"] * 1e-3
    nb = np.asarray(ens["n_body"])
    steps = steps_by_system(ens, state, dt)
    per_n = {int(n): float(scope_hermite_flops(int(n)) * steps[nb == n].sum()) for n in np.unique(nb)}
    flops = sum(per_n.values())
    return {"system_steps_per_s": st["system_steps"] / sec, "pair_interactions_per_s": st["pair_evaluations"] / sec,
            "kernel_ms": st["kernel_ms"], "launches": st["kernel_launches"], "system_steps": st["system_steps"],
            "kepler_iterations": 0, "fp64_flops": flops, "fp64_tflops": flops / sec / 1e12, "fp64_frac": flops / sec / peak,
            "fp64_count": "scope table: 3 P 58 + 3 n 34 per Hermite step",
            "fp64_flops_share_by_n": {n: f / flops for n, f in per_n.items()}}


def bins_alone(S, stream, ens, steps, dt, peak):
    """Each body count's systems integrated by themselves (one single-bin launch, `steps`
    fixed steps): system-steps/s and FP64 fraction per n by the scope table's count.  A
    bin alone runs in whole waves of its groups, which the concurrent launches hide."""
    import numpy as np

    from paper_1208_1157_gb300 import ics

    nb = np.asarray(ens["n_body"])
    out = {}
    for n in np.unique(nb):
        sub = ics.subset(ens, np.flatnonzero(nb == n))
        r = timed_per_bin(S, stream, sub, steps * dt, dt, peak)
        out[int(n)] = {"systems": int(np.sum(nb == n)), "system_steps_per_s": r["system_steps_per_s"],
                       "fp64_frac": r["fp64_frac"]}
    return out


def served_flops(trace, results):
    """FP64 work of served requests by the scope table's counts (Hermite, MVS-DH with one
    Newton iteration per drift), from the steps each system took."""
    import numpy as np

    tot = 0.0
    for r, q in enumerate(trace):
        res = results[r]
        dt = DT if q["integrator"] == 1 else TWO_PI / 20
        steps = np.round(np.asarray(res["time"]) / dt)
        f = scope_hermite_flops(q["n"]) if q["integrator"] == 1 else scope_mvs_flops(q["n"], 1.0, False)
        tot += f * float(steps.sum())
    return tot


def serving(S, stream, peak, n_req=512, rate=200.0, scales=((2000.0, 16384), (1000.0, 16384), (100.0, 4096)),
            quantum=200):
    """Continuous batching on the bounded Poisson trace (512 requests at 200/s, sizes
    log-U 1..4096, n ~ U{3..15}, Hermite / MVS-DH 50/50).  The trace's t_end (10..10^4
    inner periods) offers ~10^3 times the GPU's FP64 capacity, so it is replayed with
    t_end divided by each load scale, with pools of the given slots (at 100 and 4096 slots
    per pool, systems queue for slots); latency = submit to retirement of the request's
    last system (wall clock)."""
    from paper_1208_1157_gb300 import ics
    from paper_1208_1157_gb300 import server as SV

    res = {}
    for F, slots in scales:
        trace = ics.serving_trace(n_req=n_req, seed=5, rate=rate, t_scale=F)
        ens = [ics.request_ensemble(q) for q in trace]
        with SV.Server(slots_per_pool=slots, quantum_steps=quantum, stream=stream) as sv:
            # warm-up: the autotuner measures each (integrator, n) pool shape once
            warm = [dict(q, arrival_s=0.0, t_end=q["t_end"] * 1e-3) for q in trace[:32]]
            SV.replay(sv, warm, ens[:32])
            base = sv.stats()
            out = SV.replay(sv, trace, ens, collect=True)
            st = sv.stats()
        lat = sorted(d["latency_s"] for d in out["done"].values())
        steps = st["system_steps"] - base["system_steps"]
        kms = st["kernel_ms"] - base["kernel_ms"]
        occ = out["occupancy"]
        flops = served_flops(trace, out["done"])
        res[f"t_end_divided_by_{int(F)}"] = {
            "requests": n_req, "rate_per_s": rate, "slots_per_pool": slots, "p50_latency_s": lat[len(lat) // 2],
            "p99_latency_s": lat[min(len(lat) - 1, int(0.99 * len(lat)))], "max_latency_s": lat[-1],
            "wall_s": out["wall_s"], "system_steps": steps, "system_steps_per_s": steps / out["wall_s"],
            "gpu_busy_fraction": kms / 1e3 / out["wall_s"], "quanta": st["quanta"] - base["quanta"],
            "max_queued": max(o[2] for o in occ), "max_occupied_slots": max(o[1] for o in occ),
            "fp64_flops": flops, "fp64_frac_of_wall": flops / out["wall_s"] / peak,
            "fp64_frac_of_kernel_time": flops / (kms * 1e-3) / peak,
            "fp64_count": "scope table (Hermite; MVS-DH at one Newton iteration per drift)"}
    return res


def serving_by_integrator(S, stream, peak, F=1000.0, quantum=200):
    """Attribution of the served FP64 fraction: the t_end / F trace split into its Hermite
    and its MVS-DH requests, each half served alone with all its requests present at the
    start (closed loop), FP64 work by the scope table's counts over kernel time.  The mix
    lands between the two halves, weighted by their kernel time."""
    from paper_1208_1157_gb300 import ics
    from paper_1208_1157_gb300 import server as SV

    full = ics.serving_trace(n_req=512, seed=5, rate=200.0, t_scale=F)
    out = {}
    for name, integ in (("hermite", 1), ("mvs_dh", 2)):
        trace = [dict(q, arrival_s=0.0) for q in full if q["integrator"] == integ]
        ens = [ics.request_ensemble(q) for q in trace]
        with SV.Server(slots_per_pool=16384, quantum_steps=quantum, stream=stream) as sv:
            warm = [dict(q, t_end=q["t_end"] * 1e-3) for q in trace[:16]]
            SV.replay(sv, warm, ens[:16])
            base = sv.stats()
            r = SV.replay(sv, trace, ens, collect=True)
            st = sv.stats()
        steps = st["system_steps"] - base["system_steps"]
        kms = st["kernel_ms"] - base["kernel_ms"]
        flops = served_flops(trace, r["done"])
        out[name] = {"requests": len(trace), "system_steps": steps, "kernel_ms": kms, "wall_s": r["wall_s"],
                     "system_steps_per_s_kernel": steps / (kms * 1e-3), "fp64_flops": flops,
                     "fp64_frac_of_kernel_time": flops / (kms * 1e-3) / peak}
    return out


def serving_vs_plain(S, stream, peak, F=1000.0, quantum=200):
    """The same work three ways, all requests present at the start (closed loop, as fast as
    the GPU goes): the Hermite requests with n <= 8 of the t_end / 1000 trace (the plain
    kernel exists for n <= 8) served by continuous batching, run one after another through
    the plain one-launch-per-step kernel, and one after another through the persistent
    single-bin kernel.  system-steps/s on wall time (host work included) and on kernel time."""
    import numpy as np

    from paper_1208_1157_gb300 import ics
    from paper_1208_1157_gb300 import server as SV

    trace = [dict(q, arrival_s=0.0) for q in ics.serving_trace(n_req=512, seed=5, rate=200.0, t_scale=F)
             if q["integrator"] == 1 and q["n"] <= 8]
    ens = [ics.request_ensemble(q) for q in trace]
    out = {"requests": len(trace), "systems": int(sum(q["n_sys"] for q in trace))}
    with SV.Server(slots_per_pool=16384, quantum_steps=quantum, stream=stream) as sv:
        warm = [dict(q, t_end=q["t_end"] * 1e-3) for q in trace[:16]]
        SV.replay(sv, warm, ens[:16])
        base = sv.stats()
        r = SV.replay(sv, trace, ens, collect=True)
        st = sv.stats()
    steps = st["system_steps"] - base["system_steps"]
    kms = st["kernel_ms"] - base["kernel_ms"]
    flops = served_flops(trace, r["done"])
    out["served"] = {"wall_s": r["wall_s"], "kernel_ms": kms, "system_steps": steps,
                     "system_steps_per_s_wall": steps / r["wall_s"], "system_steps_per_s_kernel": steps / (kms * 1e-3),
                     "fp64_frac_of_wall": flops / r["wall_s"] / peak}
    for name, mapping in (("plain_one_launch_per_step", S.MAP_PLAIN_PER_STEP), ("persistent_alone", 0)):
        steps = 0
        kms = 0.0
        torch_sync = __import__("torch").cuda.synchronize
        torch_sync()
        t0 = time.perf_counter()
        for q, e in zip(trace, ens):
            with S.Ensemble(e, stream=stream) as en:
                en.set_option(S.OPT_MAPPING, mapping)
                en.set_stop(3.0, 100.0)
                en.integrate(q["t_end"], S.HERMITE4, DT)
                s_ = en.stats()
            steps += s_["system_steps"]
            kms += s_["kernel_ms"]
        torch_sync()
        wall = time.perf_counter() - t0
        out[name] = {"wall_s": wall, "kernel_ms": kms, "system_steps": steps, "system_steps_per_s_wall": steps / wall,
                     "system_steps_per_s_kernel": steps / (kms * 1e-3), "fp64_frac_of_wall": flops / wall / peak}
    out["served_over_plain_wall"] = out["served"]["system_steps_per_s_wall"] / out["plain_one_launch_per_step"]["system_steps_per_s_wall"]
    return out


def run_ours(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # CPU baseline first: the oracle's process pool is spawned before any CUDA use
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_throughput(target_s=args.cpu_seconds)
        log(f"cpu baseline: {cpu['value']:.3e} system-steps/s on {cpu['cores']} cores")
        if not args.no_secondary:
            cpu["single_core_by_workload"] = oracle_config_rates()

    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1208_1157_gb300 import ics
    from paper_1208_1157_gb300 import swarm as S

    stream = torch.cuda.current_stream()
    # the autotuner's saved choices for this GPU (paper_1208_1157_gb300/tune.py): the same
    # decisions with or without a profiler attached
    from paper_1208_1157_gb300 import tune
    S.tuner_load(tune.DEFAULT_PATH)
    pclk = Clocks(local)  # the probe's own clocks: the peak is only as good as them
    pclk.start()
    peak = S.fp64_peak(1.0, stream)
    peak_clocks = pclk.stop()
    log(f"measured FP64 peak {peak / 1e12:.4f} TFLOP/s at {peak_clocks.get('sm_mhz')} MHz")
    ens = ics.three_body(N_SYS, seed=rank_seed(rank))
    T = STEPS_PER_CALL * DT
    e = S.Ensemble(ens, stream=stream)
    e.set_stop(3.0, 100.0)
    e.set_option(S.OPT_LOG_CAPACITY, 64)
    e.set_option(S.OPT_LOG_INTERVAL, LOG_EVERY)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > 129 MB L2
    t = 0.0
    for _ in range(args.warmup):
        t += T
        e.integrate(t, S.HERMITE4, DT)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = Clocks(local)
    clocks.start()
    barrier()
    t0 = time.perf_counter()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    steps_done = pairs_done = 0
    kernel_ms = []
    for k in range(args.steps):
        flush.zero_()
        t += T
        ev[k][0].record(stream)
        e.integrate(t, S.HERMITE4, DT)
        ev[k][1].record(stream)
        st = e.stats()
        steps_done += st["system_steps"]
        pairs_done += st["pair_evaluations"]
        kernel_ms.append(st["kernel_ms"])
    barrier()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    if dist:
        (ms,), (steps_total, pairs_total) = reduce_over_ranks(dist, [ms], [steps_done, pairs_done], "cuda")
    else:
        steps_total, pairs_total = float(steps_done), float(pairs_done)
    sec = ms * 1e-3
    value = steps_total / sec

    # ---- end to end through the C ABI with pinned host buffers, copies inside the region
    pos_h = torch.empty((e.n_bodies, 3), dtype=torch.float64, pin_memory=True).numpy()
    vel_h = torch.empty((e.n_bodies, 3), dtype=torch.float64, pin_memory=True).numpy()
    tim_h = torch.empty(e.n_sys, dtype=torch.float64, pin_memory=True).numpy()
    sta_h = torch.empty(e.n_sys, dtype=torch.int32, pin_memory=True).numpy()
    e.state_into(pos_h, vel_h, tim_h, sta_h)
    barrier()
    e2e_t0 = time.perf_counter()
    e2e_steps = 0
    for k in range(args.steps):
        flush.zero_()
        t += T
        e.set_state(pos_h, vel_h, tim_h, sta_h)
        e.integrate(t, S.HERMITE4, DT)
        e2e_steps += e.stats()["system_steps"]
        e.state_into(pos_h, vel_h, tim_h, sta_h)
    barrier()
    e2e_wall = time.perf_counter() - e2e_t0
    if dist:
        (e2e_wall,), (e2e_steps,) = reduce_over_ranks(dist, [e2e_wall], [e2e_steps], "cuda")
    bytes_io = pos_h.nbytes + vel_h.nbytes + tim_h.nbytes + sta_h.nbytes

    fl = scope_hermite_flops(N_BODY)  # the scope table's count (828 at n = 3)
    fl_impl = hermite_flops_per_system_step(N_BODY)  # the implemented star-relative form (633)
    launch_ms = statistics.mean(kernel_ms)
    flops_per_launch = fl * steps_done / args.steps
    achieved = flops_per_launch / (launch_ms * 1e-3)
    achieved_impl = fl_impl * steps_done / args.steps / (launch_ms * 1e-3)
    traffic = traffic_per_launch("hermite_uniform_kernel", N_SYS)
    sec_out = {}
    if rank == 0 and not args.no_secondary:
        sec_out = secondary(S, torch, stream, peak)
    e.close()
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "system-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded planetary ICs, no dataset)",
        "config": {"workload": WORKLOAD, "n_sys_per_gpu": N_SYS, "n_body": N_BODY, "steps_per_call": STEPS_PER_CALL,
                   "dt": DT, "l2": "256 MB buffer written before every timed step (state is 22 MB < L2)",
                   "parallelism": f"replicas x{world} (independent ensembles, no collective)"},
        "pair_interactions_per_s": pairs_total / sec,
        "fp64_flops_per_system_step": fl,
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "hermite_uniform_kernel<system per lane, n=3>",
                     "flops_per_system_step": fl,
                     "flops_count": "scope table: 3 P 58 + 3 n 34 (n = 3: 828), the inertial step as the method states it",
                     "frac_implemented_form": achieved_impl / peak,
                     "flops_per_system_step_implemented_form": fl_impl,
                     "implemented_form": "star-relative coordinates with the barycentre's drift: the same map in exact "
                                         "arithmetic with fewer operations (633 at n = 3)",
                     "peak_kind": "measured DFMA-chain peak on this GPU (2 flops per DFMA), of measured",
                     "peak_clocks": peak_clocks,
                     "avg_launch_ms": launch_ms},
        "e2e": {"value": e2e_steps / e2e_wall, "unit": "system-steps/s", "h2d_bytes_per_step": bytes_io,
                "d2h_bytes_per_step": bytes_io},
        "gpu_launches": args.steps,
        "clocks": clk,
        "cpu_baseline": cpu,
        "paper_context": {"system_steps_per_s_tesla_c2070_derived": 4.47e6,
                          "note": "131072 x 3 Hermite, Table 3, 1 time unit at dt=1e-3; other hardware"},
        "secondary": sec_out,
    }
    print(json.dumps(line), flush=True)


def ncu_case(name):
    """One small fixed run of a kernel, for Nsight Compute captures (no timing)."""
    import torch

    from paper_1208_1157_gb300 import ics
    from paper_1208_1157_gb300 import swarm as S

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    from paper_1208_1157_gb300 import tune
    S.tuner_load(tune.DEFAULT_PATH)
    if name in ("io", "io_large"):  # checkpoint I/O: set_state + state query, 3 times
        import numpy as np

        # io: the paper-shaped ensemble (the state fits in L2); io_large: 16x as many
        # systems (2^21 x 3, 330 MB of state), a transfer long enough for steady bandwidth
        ns = N_SYS if name == "io" else 16 * N_SYS
        ens = ics.three_body(ns, seed=2)
        pos = torch.empty((len(ens["mass"]), 3), dtype=torch.float64, pin_memory=True).numpy()
        vel = torch.empty_like(torch.from_numpy(pos)).pin_memory().numpy()
        # the same bytes moved by a plain elementwise kernel (read a, write b = 1.0 * a):
        # the ceiling for a transfer of this size
        a = torch.ones(len(ens["mass"]) * 6, dtype=torch.float64, device="cuda")
        b = torch.empty_like(a)
        with S.Ensemble(ens, stream=stream) as e:
            for _ in range(3):
                e.set_state(ens["pos"], ens["vel"])
                e.state_into(pos, vel, np.empty(ns), np.empty(ns, np.int32))
                torch.mul(a, 1.0, out=b)
        torch.cuda.synchronize()
        log(f"ncu case {name}: {ns} systems x {N_BODY} bodies")
        return
    ctas = 0
    if name in ("hermite", "hermite_bpl", "plain"):
        ens = ics.three_body(N_SYS, seed=2)
        mapping = {"hermite": S.MAP_SYSTEM_PER_LANE, "hermite_bpl": S.MAP_BODY_PER_LANE, "plain": S.MAP_PLAIN_PER_STEP}[name]
        steps, integ, dt = (200 if name != "plain" else 20), S.HERMITE4, DT
    elif name in ("mvs", "mvs_2cta"):
        ens = ics.mvs_compact(16384, seed=4)
        mapping, steps, integ, dt = S.MAP_BODY_PER_LANE, 200, S.MVS_JACOBI, TWO_PI / 20
        ctas = 2 if name == "mvs_2cta" else 0
    elif name == "ragged":  # the 65536-system ragged ensemble as the benchmark runs it, 200 steps
        ens = ics.ragged(65536, seed=3)
        mapping, steps, integ, dt = S.MAP_AUTO, 200, S.HERMITE4, DT
    elif name.startswith("ragged_bin"):  # one body count of the ragged set (default n = 13), 100 steps
        import numpy as np

        n = int(name[len("ragged_bin"):] or 13)
        full = ics.ragged(65536, seed=3)
        ens = ics.subset(full, np.flatnonzero(np.asarray(full["n_body"]) == n))
        mapping, steps, integ, dt = S.MAP_BODY_PER_LANE, 100, S.HERMITE4, DT
    elif name == "rkck":
        ens = ics.three_body(N_SYS, seed=2)
        mapping, steps, integ, dt = S.MAP_BODY_PER_LANE, 50, S.RKCK, DT
    elif name == "hermite_adaptive":  # Eq. 5 steps, tau = 0.01, over 1/10 inner period
        ens = ics.three_body(N_SYS, seed=2)
        mapping, steps, integ, dt = S.MAP_SYSTEM_PER_LANE, 1, S.HERMITE4_ADAPTIVE, 0.01
    elif name == "rkck_adaptive":  # error-controlled steps, tolerance 1e-12, over 1/10 inner period
        ens = ics.three_body(N_SYS, seed=2)
        mapping, steps, integ, dt = S.MAP_BODY_PER_LANE, 1, S.RKCK_ADAPTIVE, 0.05
    elif name == "wide":
        ens = ics.ragged_wide(16384, seed=6)
        mapping, steps, integ, dt = S.MAP_AUTO, 10, S.HERMITE4, DT
    else:
        raise SystemExit(f"unknown case {name}")
    with S.Ensemble(ens, stream=stream) as e:
        e.set_option(S.OPT_MAPPING, mapping)
        e.set_option(S.OPT_CTAS_PER_SM, ctas)
        e.set_stop(3.0, 100.0)
        t_end = 0.1 * TWO_PI if integ in (S.HERMITE4_ADAPTIVE, S.RKCK_ADAPTIVE) else steps * dt
        e.integrate(t_end, integ, dt)
        st = e.stats()
    log(f"ncu case {name}: {st}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--ncu-case", help="hermite, hermite_bpl, plain, mvs, mvs_2cta, ragged, ragged_bin<n>, rkck, wide, "
                    "hermite_adaptive, rkck_adaptive, io or io_large")
    args = ap.parse_args()
    if args.ncu_case:
        ncu_case(args.ncu_case)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
