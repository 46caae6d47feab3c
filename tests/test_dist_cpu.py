"""The multi-rank (replica) path of bench.py on CPU: two gloo ranks run the same
aggregation code the GPU ranks run (max of the per-rank times over all ranks, whole-job
units), and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, q) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    ms, value = bench.combine_ranks(10.0 * (rank + 1), 40, w, "cpu")
    dist.barrier()
    q.put((rank, r, w, ms, value, bench.reference_runs_here(r)))
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, r, w, ms, value, ref_here in res:
        assert r == rank and w == 2
        assert ms == 20.0  # the slowest rank's time, on every rank
        assert value == pytest.approx(40 * 2 / 0.020)  # units of both ranks / max time
        assert ref_here == (rank == 0)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.combine_ranks(5.0, 10, 1)
    assert ms == 5.0 and value == pytest.approx(2000.0)
