"""The multi-rank host logic of bench.py on CPU: two ranks over gloo
(127.0.0.1) agree on the slowest rank's time, the whole-job throughput counts
every rank's environments (weak scaling: environments shard by rank, no
data-path collective), each rank draws its own seeded workload, and the
reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    from paper_2509_10247_b300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, world)
        p = synth.preset("swarm_16384env_8agent_8maps_depth16x9", n_env=4)
        s0 = synth.make_inputs(p, seed=0 + rank)["s0"]
        out[rank] = (ms, bench.job_throughput(4, 64, 3, world, ms), s0[:2].tolist())
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_max_time_and_count_all_environments():
    world, port = 2, _port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    (ms0, v0, s_a), (ms1, v1, s_b) = res[0], res[1]
    assert ms0 == ms1 == 15.0
    assert v0 == v1 == 4 * 64 * 3 * 2 / 0.015
    assert not np.allclose(s_a, s_b)  # each rank its own environments


def test_reference_arm_runs_on_rank_zero_only():
    # ranks other than 0 exit 0 without work and print nothing
    env = dict(os.environ, RANK="1", WORLD_SIZE="1", LOCAL_RANK="1")
    code = ("import sys; sys.path.insert(0, %r); import bench; "
            "a = bench.parse(); print(bench.run_reference(a, 1, 2))") % ROOT
    r = subprocess.run([sys.executable, "-c", code, "--impl", "reference"], env=env, capture_output=True,
                       text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert not lines
