"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): timings reduce to the
maximum over ranks, the whole-job rate counts every rank's queries, each rank searches
its own deterministic query batch, and the reference arm does no work off rank 0."""

import os
import subprocess
import sys

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dev_s, e2e_s = bench.max_over_ranks([1.0 + rank, 5.0 - rank], world, "cpu")
    out[rank] = (dev_s, e2e_s, bench.whole_job_rate(100, world, dev_s))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    world, port = 2, 29500 + os.getpid() % 1000
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        assert out[r][0] == 2.0 and out[r][1] == 5.0     # the slowest rank on both counts
        assert out[r][2] == 100.0                         # 2 ranks x 100 units / 2 s


def test_rank_queries_are_distinct_and_deterministic():
    import bench
    q0, q1 = bench.rank_queries(0), bench.rank_queries(1)
    assert q0.shape == q1.shape == (bench.NQ, bench.D)
    assert not np.allclose(q0, q1)
    assert np.array_equal(q1, bench.rank_queries(1))


def test_reference_arm_does_nothing_off_rank_zero():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
