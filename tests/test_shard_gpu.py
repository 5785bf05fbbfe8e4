"""The i-sharded path with libfsi as the shard compute (LibfsiCompute) on the GPU.

Two gloo ranks share cuda:0 (independent contexts and kernels; no kernel waits on the other
rank, the exchange goes through host memory), and one NCCL rank runs the same path through
NCCL collectives; both against the oracle and the one-rank library calls: the pair sums of
a set, FSI cycles with PN kicks, and an HHS interval with every level's list sharded.  A
third run takes the same-set passes split by pairs (fsi_accel_part / fsi_grad_part, shares
all-reduced), the pair sums on a set of 13001 that the symmetric kernel splits.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_2210_02472_b300 import inputs

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, backend, out, pairs):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    torch.cuda.set_device(0)
    dist.init_process_group(backend, rank=rank, world_size=world)
    from paper_2210_02472_b300 import fsi as F
    from paper_2210_02472_b300.shard import LibfsiCompute, ShardedFSI
    try:
        res = {}
        for prec in ("fp64", "mixed"):
            with F.Context(prec) as ctx:
                sh = ShardedFSI(LibfsiCompute(ctx), min_rows=64, pairs=pairs)
                c = inputs.plummer(13001 if pairs else 3001, 61, imf="kroupa")
                a, g = sh.accel_grad(torch.as_tensor(c.pos).cuda(), torch.as_tensor(c.mass).cuda())
                res[prec + "_ag"] = (a.cpu().numpy(), g.cpu().numpy())
                c = inputs.plummer(900, 62, imf="kroupa", n_bh=3)
                pos, vel = torch.as_tensor(c.pos).cuda(), torch.as_tensor(c.vel).cuda()
                sh.step(pos, vel, torch.as_tensor(c.mass).cuda(), 1e-3, nsteps=3, c=40.0,
                        is_bh=torch.as_tensor(c.is_bh.astype(np.uint8)).cuda())
                torch.cuda.synchronize()
                assert F.fsi_sync_status(ctx) == F.FSI_OK
                res[prec + "_step"] = (pos.cpu().numpy(), vel.cpu().numpy())
                c = inputs.plummer(1500, 63, imf="kroupa")
                pos, vel = torch.as_tensor(c.pos).cuda(), torch.as_tensor(c.vel).cuda()
                counts, hit = sh.hhs_interval(pos, vel, torch.as_tensor(c.mass).cuda(), 1.0 / 32)
                torch.cuda.synchronize()
                assert F.fsi_sync_status(ctx) == F.FSI_OK and not hit
                res[prec + "_hhs"] = (pos.cpu().numpy(), vel.cpu().numpy(), np.array(counts))
        out[rank] = res
    finally:
        dist.destroy_process_group()


def _run(world, backend, pairs=False):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, backend, out, pairs))
                 for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(900)
            assert p.exitcode == 0, f"rank exited with {p.exitcode}"
        return [out[r] for r in range(world)]


def _check(outs, n_ag=3001):
    oracle.set_threads(os.cpu_count() or 1)
    c = inputs.plummer(n_ag, 61, imf="kroupa")
    ra, rg = oracle.accel_grad(c.pos, c.mass)
    d = inputs.plummer(900, 62, imf="kroupa", n_bh=3)
    rp, rv = oracle.fsi_step(d.pos, d.vel, d.mass, 1e-3, c=40.0, is_bh=d.is_bh, steps=3)
    na, ng = np.linalg.norm(ra, axis=0), np.linalg.norm(rg, axis=0)
    e = inputs.plummer(1500, 63, imf="kroupa")
    hp, hv, hc, _ = oracle.hhs_interval(e.pos, e.vel, e.mass, 1.0 / 32)
    used = np.nonzero(hc)[0].max() + 1
    for res in outs:
        a, g = res["fp64_ag"]
        assert (np.abs(a - ra).max(axis=0) / na).max() <= 1e-12
        assert (np.abs(g - rg).max(axis=0) / ng).max() <= 1e-12
        p, v = res["fp64_step"]
        assert np.abs(p - rp).max() <= 1e-12 and np.abs(v - rv).max() <= 1e-10
        a, g = res["mixed_ag"]
        assert np.median(np.linalg.norm(a - ra, axis=0) / na) <= 1e-7
        assert np.median(np.linalg.norm(g - rg, axis=0) / ng) <= 1e-5
        p, v = res["mixed_step"]
        assert np.abs(p - rp).max() <= 1e-9 and np.abs(v - rv).max() <= 1e-7
        for prec, tol in (("fp64", 1e-11), ("mixed", 1e-7)):
            p, v, lv = res[prec + "_hhs"]
            assert list(lv[:used]) == list(hc[:used])
            assert np.abs(p - hp).max() <= tol and np.abs(v - hv).max() <= 100 * tol
    for k in outs[0]:
        for x, y in zip(outs[0][k], outs[-1][k]):
            assert np.array_equal(x, y), k          # every rank ends with the same data


def test_sharded_libfsi_two_gloo_ranks_on_one_gpu():
    _check(_run(2, "gloo"))


def test_sharded_libfsi_one_nccl_rank():
    _check(_run(1, "nccl"))


def test_sharded_libfsi_pairs_two_gloo_ranks_on_one_gpu():
    _check(_run(2, "gloo", pairs=True), n_ag=13001)
