"""The N > 1 path of the benchmark on CPU: two gloo ranks.

Systems are independent, so ranks share no data; each integrates its own seeded
ensemble (here with the CPU oracle standing in for the device work), and only the
timing reduction (max of times, sum of work over ranks) crosses ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle as O
    from paper_1208_1157_gb300 import ics

    ens = ics.three_body(8, seed=bench.rank_seed(rank))
    o = O.integrate(ens, 20 * bench.DT, bench.DT, O.HERMITE)
    steps = int(np.sum(np.round(o["time"] / bench.DT)))
    ms = 10.0 + rank  # per-rank "time"
    (mx,), (sm,) = bench.reduce_over_ranks(dist, [ms], [steps], "cpu")
    out[rank] = (mx, sm, float(o["pos"][1, 0]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_stay_independent():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    r0, r1 = out[0], out[1]
    assert r0[0] == r1[0] == 11.0            # max of the ranks' times
    assert r0[1] == r1[1] == 2 * 8 * 20       # system-steps summed over ranks
    assert r0[2] != r1[2]                     # different, independent ensembles
