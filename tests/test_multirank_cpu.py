"""The multi-rank path on CPU: two gloo ranks (world size 2).

bench.py gives each rank its own shot range and combines only timings (MAX).
These tests run that host logic with the oracle as the decoder: the ranges are
disjoint and cover the whole job, the summed failure count of the two ranks
equals one process decoding every shot (draws are keyed by the absolute shot
index, so the partition cannot change a result), and the MAX reduction is the
slowest rank's time.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STEPS, S = 2, 15


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist

    import bench
    import oracle as O
    dist.init_process_group("gloo", rank=rank, world_size=world)
    base = bench.rank_shot_base(rank, STEPS, S)
    pxyz = O.noise_from_eta(0.12, 1.0, O.PAPER_ETA)
    err, syn = O.sample(3, pxyz, 5, base, STEPS * S)
    out = O.decode(3, pxyz, 1024, O.LINEAR, 40, 0.1, 10.0, 5, base, 4, syn, err)
    fails = bench.sum_over_ranks([float(out["fail"].sum())], dist, "cpu")
    slowest = bench.max_over_ranks([1.0 + rank, 5.0 - rank], dist, "cpu")
    np.save(os.path.join(out_dir, "rank%d.npy" % rank),
            np.array([base, fails[0], slowest[0], slowest[1]], dtype=np.float64))
    dist.destroy_process_group()


def test_two_gloo_ranks_match_one_process(tmp_path):
    import oracle as O
    world, port = 2, _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn")
    r = [np.load(tmp_path / ("rank%d.npy" % k)) for k in range(world)]
    bases = sorted(int(x[0]) for x in r)
    assert bases == [0, STEPS * S]                      # disjoint ranges covering the job
    pxyz = O.noise_from_eta(0.12, 1.0, O.PAPER_ETA)
    err, syn = O.sample(3, pxyz, 5, 0, world * STEPS * S)
    ref = O.decode(3, pxyz, 1024, O.LINEAR, 40, 0.1, 10.0, 5, 0, 4, syn, err)
    for x in r:
        assert int(x[1]) == int(ref["fail"].sum())     # summed failures: partition-independent
        assert x[2] == 2.0 and x[3] == 5.0              # MAX over ranks
