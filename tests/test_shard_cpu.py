"""The i-sharded exchange layer (paper_2210_02472_b300.shard) on gloo ranks on the CPU.

The shard compute is the FP64 oracle here (the product plugs libfsi in), so these tests
check what the exchange layer adds: the slicing of the active list, the all-gathers of
positions after drifts and of accelerations before the gradient pass, the source split
with an all-reduce for small active sets, and the kick/drift bookkeeping of the FSI cycle
-- against the same computation on one rank (the oracle called directly), which they must
match up to summation order.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_2210_02472_b300 import inputs
from paper_2210_02472_b300.shard import ShardedFSI, slice_bounds


class OracleCompute:
    """Shard compute on CPU tensors through the FP64 oracle."""

    def accel(self, pos, mass, A, B, eps2):
        return torch.as_tensor(oracle.acc(pos.numpy(), mass.numpy(), A.numpy(), B.numpy(), eps2))

    def grad(self, pos, mass, accg, A, B, eps2):
        return torch.as_tensor(oracle.grad(pos.numpy(), mass.numpy(), accg.numpy(), A.numpy(),
                                           B.numpy(), eps2))

    # a share of a same-set pass: the receivers against slice `part` of the sources (any
    # partition of the pairs serves the exchange; libfsi's shares are blocks of its
    # symmetric kernel)
    def accel_part(self, pos, mass, A, part, nparts, eps2):
        lo, hi = slice_bounds(A.numel(), nparts, part)
        return self.accel(pos, mass, A, A[lo:hi].contiguous(), eps2)

    def grad_part(self, pos, mass, accg, A, part, nparts, eps2):
        lo, hi = slice_bounds(A.numel(), nparts, part)
        return self.grad(pos, mass, accg, A, A[lo:hi].contiguous(), eps2)

    def pn_accel(self, pos, vel, mass, is_bh, c, A, B):
        return torch.as_tensor(oracle.pn_acc(pos.numpy(), vel.numpy(), mass.numpy(), is_bh.numpy(),
                                             c, A.numpy(), B.numpy()))

    def kick_drift(self, pos, vel, acc, idx, c_kick, c_drift):
        p, v = oracle.kick_drift(pos.numpy(), vel.numpy(), None if acc is None else acc.numpy(),
                                 c_kick, c_drift, idx.numpy())
        pos.copy_(torch.as_tensor(p))
        vel.copy_(torch.as_tensor(v))

    def timesteps(self, pos, vel, mass, P, eps2):
        return torch.as_tensor(oracle.timesteps(pos.numpy(), vel.numpy(), mass.numpy(), P.numpy(),
                                                eps2=eps2))

    def timesteps_rows(self, pos, vel, mass, P, lo, hi, eps2):
        return self.timesteps(pos, vel, mass, P, eps2)[lo:hi]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, case, out):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    oracle.set_threads(1)
    try:
        name, _, mode = case.partition("+")
        out[rank] = CASES[name](ShardedFSI(OracleCompute(), min_rows=16, pairs=mode == "pairs"))
    finally:
        dist.destroy_process_group()


def _run(case, world):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, case, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0, f"rank exited with {p.exitcode}"
        return [out[r] for r in range(world)]


# ---------------------------------------------------------------- cases (run on every rank)
def _same_set(sh):
    c = inputs.plummer(701, 51, imf="kroupa")
    a, g = sh.accel_grad(torch.as_tensor(c.pos), torch.as_tensor(c.mass))
    return a.numpy(), g.numpy()


def _disjoint_softened(sh):
    c = inputs.plummer(640, 52, imf="kroupa")
    perm = np.random.default_rng(53).permutation(640).astype(np.int32)
    S, F = torch.as_tensor(np.sort(perm[:500])), torch.as_tensor(np.sort(perm[500:]))
    a, g = sh.accel_grad(torch.as_tensor(c.pos), torch.as_tensor(c.mass), S, F, eps2=1e-4)
    return a.numpy(), g.numpy()


def _small_set_split_sources(sh):
    c = inputs.plummer(400, 54, imf="kroupa")
    A = torch.as_tensor(np.array([3, 17, 99, 250, 391], dtype=np.int32))   # 5 < 16 x ranks
    a, g = sh.accel_grad(torch.as_tensor(c.pos), torch.as_tensor(c.mass), A, A)
    return a.numpy(), g.numpy()


def _steps(sh):
    c = inputs.plummer(301, 55, imf="kroupa")
    pos, vel = torch.as_tensor(c.pos.copy()), torch.as_tensor(c.vel.copy())
    sh.step(pos, vel, torch.as_tensor(c.mass), 1e-3, nsteps=3)
    return pos.numpy(), vel.numpy()


def _steps_subset_pn(sh):
    c = inputs.plummer(260, 56, imf="kroupa", n_bh=4)
    P = np.sort(inputs.random_subset(260, 150, 57)).astype(np.int32)
    P = np.union1d(P, np.nonzero(c.is_bh)[0]).astype(np.int32)
    pos, vel = torch.as_tensor(c.pos.copy()), torch.as_tensor(c.vel.copy())
    sh.step(pos, vel, torch.as_tensor(c.mass), 1e-3, nsteps=2, idx=torch.as_tensor(P), c=30.0,
            is_bh=torch.as_tensor(c.is_bh.astype(np.uint8)))
    return pos.numpy(), vel.numpy()


def _hhs(sh):
    c = inputs.plummer(300, 58, imf="kroupa")
    pos, vel = torch.as_tensor(c.pos.copy()), torch.as_tensor(c.vel.copy())
    counts, hit = sh.hhs_interval(pos, vel, torch.as_tensor(c.mass), 1.0 / 16)
    return pos.numpy(), vel.numpy(), counts, hit


def _hhs_pn_softened_capped(sh):
    c = inputs.plummer(240, 59, imf="kroupa", n_bh=4)
    pos, vel = torch.as_tensor(c.pos.copy()), torch.as_tensor(c.vel.copy())
    counts, hit = sh.hhs_interval(pos, vel, torch.as_tensor(c.mass), 1.0 / 16, eps2=1e-5, c=30.0,
                                  is_bh=torch.as_tensor(c.is_bh.astype(np.uint8)), max_level=3)
    return pos.numpy(), vel.numpy(), counts, hit


CASES = {"same": _same_set, "disjoint": _disjoint_softened, "small": _small_set_split_sources,
         "steps": _steps, "steps_pn": _steps_subset_pn, "hhs": _hhs,
         "hhs_pn": _hhs_pn_softened_capped}


# ---------------------------------------------------------------- tests
def test_slice_bounds_cover_the_list_once():
    for n in (0, 1, 5, 701, 1024):
        for w in (1, 2, 3, 8):
            b = [slice_bounds(n, w, r) for r in range(w)]
            assert b[0][0] == 0 and b[-1][1] == n
            assert all(b[k][1] == b[k + 1][0] for k in range(w - 1))
            assert max(h - l for l, h in b) - min(h - l for l, h in b) <= 1


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_accel_grad_same_set(world):
    c = inputs.plummer(701, 51, imf="kroupa")
    ra, rg = oracle.accel_grad(c.pos, c.mass)
    outs = _run("same", world)
    for a, g in outs:          # receivers split by rows: each row's sum as on one rank
        assert np.array_equal(a, ra) and np.array_equal(g, rg)


def test_sharded_accel_grad_inter_level_softened():
    c = inputs.plummer(640, 52, imf="kroupa")
    perm = np.random.default_rng(53).permutation(640).astype(np.int32)
    S, F = np.sort(perm[:500]), np.sort(perm[500:])
    ra, rg = oracle.accel_grad(c.pos, c.mass, S, F, eps2=1e-4)
    for a, g in _run("disjoint", 2):
        assert np.array_equal(a, ra) and np.array_equal(g, rg)


def test_sharded_small_set_splits_sources():
    """Five active particles on two ranks: sources split, partial sums all-reduced (the
    summation order changes, so the results agree to rounding)."""
    c = inputs.plummer(400, 54, imf="kroupa")
    A = np.array([3, 17, 99, 250, 391], dtype=np.int32)
    ra, rg = oracle.accel_grad(c.pos, c.mass, A, A)
    outs = _run("small", 2)
    for a, g in outs:
        assert np.abs(a - ra).max() <= 1e-13 * np.abs(ra).max()
        assert np.abs(g - rg).max() <= 1e-13 * np.abs(rg).max()
    assert np.array_equal(outs[0][0], outs[1][0])       # every rank holds the same sums


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_accel_grad_same_set_split_by_pairs(world):
    """pairs=True: each rank sums a share of the set's pairs for all receivers and the
    shares are all-reduced; the sums agree with the one-rank ones to rounding and are the
    same on every rank."""
    c = inputs.plummer(701, 51, imf="kroupa")
    ra, rg = oracle.accel_grad(c.pos, c.mass)
    outs = _run("same+pairs", world)
    for a, g in outs:
        assert np.abs(a - ra).max() <= 1e-13 * np.abs(ra).max()
        assert np.abs(g - rg).max() <= 1e-13 * np.abs(rg).max()
    assert all(np.array_equal(o[0], outs[0][0]) and np.array_equal(o[1], outs[0][1]) for o in outs)


@pytest.mark.parametrize("case,world", [("steps+pairs", 2), ("steps+pairs", 3), ("steps_pn+pairs", 2)])
def test_sharded_fsi_steps_split_by_pairs(case, world):
    """FSI cycles with the same-set passes split by pairs: every rank kicks and drifts the
    whole set with the all-reduced sums, so the replicas stay identical with no position
    exchange; against the one-rank oracle (the whole set, and a subset with PN1.0)."""
    if case.startswith("steps_pn"):
        c = inputs.plummer(260, 56, imf="kroupa", n_bh=4)
        P = np.sort(inputs.random_subset(260, 150, 57)).astype(np.int32)
        P = np.union1d(P, np.nonzero(c.is_bh)[0]).astype(np.int32)
        rp, rv = oracle.fsi_step(c.pos, c.vel, c.mass, 1e-3, P=P, c=30.0, is_bh=c.is_bh, steps=2)
    else:
        c = inputs.plummer(301, 55, imf="kroupa")
        rp, rv = oracle.fsi_step(c.pos, c.vel, c.mass, 1e-3, steps=3)
    outs = _run(case, world)
    for p, v in outs:
        assert np.abs(p - rp).max() <= 1e-14 * np.abs(rp).max()
        assert np.abs(v - rv).max() <= 1e-12 * np.abs(rv).max()
    assert all(np.array_equal(o[0], outs[0][0]) and np.array_equal(o[1], outs[0][1]) for o in outs)


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_fsi_steps_match_one_rank(world):
    c = inputs.plummer(301, 55, imf="kroupa")
    rp, rv = oracle.fsi_step(c.pos, c.vel, c.mass, 1e-3, steps=3)
    outs = _run("steps", world)
    for p, v in outs:
        assert np.abs(p - rp).max() <= 1e-14 * np.abs(rp).max()
        assert np.abs(v - rv).max() <= 1e-13 * np.abs(rv).max()
    assert np.array_equal(outs[0][0], outs[-1][0]) and np.array_equal(outs[0][1], outs[-1][1])


def test_sharded_fsi_steps_subset_with_pn():
    """FSI cycles of a subset with PN1.0 half-kicks (4 black holes, c = 30): particles
    outside the set do not move, and the set matches the one-rank oracle."""
    c = inputs.plummer(260, 56, imf="kroupa", n_bh=4)
    P = np.sort(inputs.random_subset(260, 150, 57)).astype(np.int32)
    P = np.union1d(P, np.nonzero(c.is_bh)[0]).astype(np.int32)
    rp, rv = oracle.fsi_step(c.pos, c.vel, c.mass, 1e-3, P=P, c=30.0, is_bh=c.is_bh, steps=2)
    for p, v in _run("steps_pn", 2):
        assert np.abs(p - rp).max() <= 1e-14 * np.abs(rp).max()
        assert np.abs(v - rv).max() <= 1e-12 * np.abs(rv).max()
        others = np.setdiff1d(np.arange(260), P)
        assert np.array_equal(p[:, others], c.pos[:, others])


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("mode", ["", "+pairs"])
def test_sharded_hhs_interval_matches_oracle(world, mode):
    """One HHS interval (Sect. 2.2) with every level's active list sharded over 2 or 3
    ranks (row slices of the inter-level kicks and the FSI(S) cycles, gathered sums; with
    "+pairs" the FSI(S) passes split by pairs instead, shares all-reduced) against the
    oracle's interval on one rank: the same level histogram, the state to rounding, and
    the same state on every rank."""
    c = inputs.plummer(300, 58, imf="kroupa")
    rp, rv, counts, code = oracle.hhs_interval(c.pos, c.vel, c.mass, 1.0 / 16)
    outs = _run("hhs" + mode, world)
    used = np.nonzero(counts)[0].max() + 1
    for p, v, lv, hit in outs:
        assert lv[:used] == list(counts[:used]) and not hit
        assert np.abs(p - rp).max() <= 1e-13
        assert np.abs(v - rv).max() <= 1e-11
    assert np.array_equal(outs[0][0], outs[-1][0]) and np.array_equal(outs[0][1], outs[-1][1])


def test_sharded_hhs_interval_pn_softened_depth_cap():
    """The sharded interval with PN1.0 S-F and S-S kicks (4 black holes, c = 30),
    softening and a depth cap of 3 levels, against the oracle's capped interval."""
    c = inputs.plummer(240, 59, imf="kroupa", n_bh=4)
    rp, rv, counts, code = oracle.hhs_interval(c.pos, c.vel, c.mass, 1.0 / 16, eps2=1e-5, c=30.0,
                                               is_bh=c.is_bh, max_level=3, allow_maxlevel=True)
    outs = _run("hhs_pn", 2)
    used = np.nonzero(counts)[0].max() + 1
    for p, v, lv, hit in outs:
        assert lv[:used] == list(counts[:used])
        assert hit and code == oracle.ERR_MAXLEVEL
        assert np.abs(p - rp).max() <= 1e-13
        assert np.abs(v - rv).max() <= 1e-11 * max(1.0, np.abs(rv).max())
