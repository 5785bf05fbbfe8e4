"""The benchmark's multi-rank path (one replica per rank, barrier, max over ranks of the
timed region, whole-job value) with two gloo ranks on CPU."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "FSI_BENCH_BACKEND": "gloo"})
    import bench
    r, ws, local, dist = bench.dist_init()
    assert (r, ws) == (rank, world)
    dist.barrier()
    t = 1.0 + rank                       # the slower rank decides the job time
    tmax = bench.reduce_max(t, dist)
    out[rank] = (tmax, bench.job_value(100.0, ws, tmax))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == out[1] == (2.0, 100.0)


def test_single_rank_is_the_identity():
    import bench
    assert bench.reduce_max(3.5, None) == 3.5
    assert bench.job_value(10.0, 1, 2.0) == 5.0
