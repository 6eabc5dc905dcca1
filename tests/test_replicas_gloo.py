"""The multi-GPU form of bench.py is independent replicas: one system per rank, no data-path collective, only a
barrier around the timed region and the maximum of the ranks' times.  These helpers run here as two gloo ranks on
the CPU (the same calls go over NCCL under torchrun on GPUs)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench

    r, ws, dist = bench.dist_init()
    assert (r, ws) == (rank, world) and dist is not None
    bench.barrier(dist)
    t = bench.max_over_ranks(dist, 10.0 * (rank + 1), "cpu")   # per-rank "step times"
    bench.barrier(dist)

    class Args:
        workload = "small"

    ref = bench.run_reference(Args(), r, ws, dist) if r != 0 else None   # non-zero ranks leave without work
    out.put((rank, t, ref))
    dist.destroy_process_group()


def test_two_rank_barrier_and_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    assert all(r[1] == 20.0 for r in res)          # every rank sees the slowest rank's time
    assert res[1][2] is None                        # the reference arm does no work off rank 0
