"""Multi-rank host logic of bench.py on CPU: two gloo ranks aggregate their
replica results (slowest rank's time, summed valid scenes), replicas draw
independent inputs, and the reference arm prints on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r: 2 + r seconds timed, 10 * (r + 1) valid scenes; e2e 3 + r seconds, 7 + r scenes
    res = bench.aggregate_ranks(2.0 + rank, 10 * (rank + 1), 3.0 + rank, 7 + rank, world, torch.device("cpu"))
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_max_time_and_summed_work():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        assert out[r] == [3.0, 30.0, 4.0, 15.0]


def test_single_rank_aggregate_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    import torch
    assert bench.aggregate_ranks(1.5, 4, 2.5, 3, 1, torch.device("cpu")) == [1.5, 4.0, 2.5, 3.0]


def test_replicas_draw_independent_inputs():
    sys.path.insert(0, ROOT)
    import bench
    import synth
    seeds = [bench.replica_seed(2, r) for r in range(4)]
    assert len(set(seeds)) == 4
    a = synth.tabletop(seed=seeds[0], n_cand=8)
    b = synth.tabletop(seed=seeds[1], n_cand=8)
    assert not (a.sph_local.shape == b.sph_local.shape and (a.sph_local == b.sph_local).all())


@pytest.mark.slow
def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--ref-step-s", "0.5", "--workload", "tabletop"],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
