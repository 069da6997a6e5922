"""Multi-GPU is "replicas only" (one independent solve per rank, no data-path
collective).  The host-side aggregation of `bench.py` is checked here on the
CPU with two gloo ranks: the whole-job iterations are the sum over the ranks
and the whole-job time is the slowest rank's, whatever the rank order."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, per_rank, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t, it = per_rank[rank]
    out.put((rank, bench.aggregate_replicas(t, it, "cpu")))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("per_rank", [[(1.5, 2377), (1.7, 2377)], [(2.25, 100), (0.5, 4000)]])
def test_replica_aggregation_two_gloo_ranks(per_rank):
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, per_rank, out)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want_t = max(t for t, _ in per_rank)
    want_it = float(sum(it for _, it in per_rank))
    for r in range(world):
        assert got[r] == (want_t, want_it)
    # the bench's value: whole-job iterations per second
    assert abs(want_it / want_t - got[0][1] / got[0][0]) < 1e-12
