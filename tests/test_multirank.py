"""The replica mode of bench.py (one process per GPU, independent query
streams, max-over-ranks timing) on two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        r, w, _ = bench.dist_env()
        # rank r timed 1 + r seconds for 10 (r + 1) queries
        elapsed, units = bench.combine_over_ranks(1.0 + r, 10 * (r + 1), w)
        seed = bench.rank_query_seed(bench.synth.CONFIGS["tiny"], r)
        out.put((r, w, elapsed, units, seed))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(180)
def test_two_ranks_max_time_and_total_units():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=150) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    # every rank sees the slowest rank's time and the queries of all ranks
    assert all(r[2] == 2.0 for r in res)
    assert all(r[3] == 30.0 for r in res)
    # the replicas draw different query streams
    assert res[0][4] != res[1][4]


def test_one_rank_passthrough():
    import bench
    assert bench.combine_over_ranks(1.5, 64, 1) == (1.5, 64.0)
