"""The multi-GPU path of bench.py, where every GPU runs its own attempts with no data-path
collective: the job's time is the slowest rank's, the throughput counts every rank's attempts,
and ranks draw disjoint inputs.  Runs as two gloo ranks on the CPU (the same calls bench.py makes
over NCCL, one process per GPU)."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench as b
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_elapsed = 2.0 + 1.5 * rank          # rank 1 is the slow one
        job = b.reduce_max(local_elapsed, world)
        value = b.job_throughput(256, 10, world, job)
        dist.barrier()
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{job} {value}\n")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_rank(tmp_path):
    world = 2
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    got = [tuple(map(float, open(tmp_path / f"rank{r}.txt").read().split())) for r in range(world)]
    for job, value in got:
        assert job == 3.5                         # the slower rank's time, seen by both ranks
        assert abs(value - 256 * 10 * 2 / 3.5) < 1e-9


def test_single_rank_needs_no_process_group():
    assert bench.reduce_max(1.25, 1) == 1.25
    assert bench.job_throughput(128, 5, 1, 2.0) == 320.0


def test_ranks_and_sets_draw_disjoint_inputs():
    seen = {}
    for rank in range(8):
        for si in range(4):
            for k in range(0, 1024, 7):
                q, n, r = bench.rank_seeds(rank, si, k)
                for kind, v in (("noise", n), ("ransac", r)):
                    assert (kind, v) not in seen, (rank, si, k, seen.get((kind, v)))
                    seen[(kind, v)] = (rank, si, k)
                assert q == bench.rank_seeds(rank, si, 0)[0]
    query_seeds = {bench.rank_seeds(r, si, 0)[0] for r in range(8) for si in range(4)}
    assert len(query_seeds) == 32
