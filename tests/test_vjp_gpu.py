"""GPU adjoint (fsi_step_vjp through the C ABI) against the oracle's adjoint, plus the
autograd wrappers: checkpointed rollouts against un-checkpointed ones and against central
finite differences of the forward."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2210_02472_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    oracle.set_threads(os.cpu_count() or 1)
    from paper_2210_02472_b300 import fsi
    return fsi


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dtype)


@pytest.mark.parametrize("n,subset", [(300, False), (1000, False), (700, True), (2500, False),
                                      (7000, True)])
def test_step_vjp_matches_oracle(F, n, subset):
    """One cycle's adjoint against the oracle's hand-derived adjoint; sets of >= 2048
    particles (2500, and the 2333 of 7000) take the symmetric adjoint pair kernels."""
    c = inputs.plummer(n, 61 + n, imf="kroupa")
    h = 1e-3
    rng = np.random.default_rng(3)
    gx, gv = rng.normal(size=(3, n)), rng.normal(size=(3, n))
    P = inputs.random_subset(n, n // 3, 5) if subset else None
    rx, rv, rm = oracle.fsi_step_vjp(c.pos, c.vel, c.mass, h, gx, gv, P=P)
    with F.Context("fp64") as ctx:
        idx = None if P is None else dev(P, torch.int32)
        gm0 = dev(np.full(n, 0.25))
        ix, iv, im = F.fsi_step_vjp(ctx, dev(c.pos), dev(c.vel), dev(c.mass), h, dev(gx), dev(gv),
                                    idx=idx, gm=gm0)
        assert F.fsi_sync_status(ctx) == F.FSI_OK
        ix, iv, im = ix.cpu().numpy(), iv.cpu().numpy(), im.cpu().numpy()
    assert np.abs(ix - rx).max() <= 1e-11 * np.abs(rx).max()
    assert np.abs(iv - rv).max() <= 1e-12 * np.abs(rv).max()
    assert np.abs(im - 0.25 - rm).max() <= 1e-11 * np.abs(rm).max()


def test_rollout_checkpointing_is_consistent(F):
    """Checkpoint spacing only changes which states are recomputed: the gradients agree
    to rounding (the symmetric pair kernels add source-side sums with FP64 atomics, so
    recomputed states can differ from the stored ones in the last bits)."""
    from paper_2210_02472_b300.autodiff import fsi_rollout
    c = inputs.plummer(400, 62)
    with F.Context("fp64") as ctx:
        grads = []
        for every in (1, 7, 50):
            x = dev(c.pos).requires_grad_(True)
            v = dev(c.vel).requires_grad_(True)
            m = dev(c.mass).requires_grad_(True)
            p, q = fsi_rollout(ctx, x, v, m, 1e-3, 12, ckpt_every=every)
            ((p * p).sum() + (q * q).sum()).backward()
            grads.append([t.grad.cpu().numpy() for t in (x, v, m)])
    for g in grads[1:]:
        for a, b in zip(g, grads[0]):
            assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max()


def test_rollout_vjp_matches_finite_differences(F):
    """L = sum |x_final|^2 after 20 FSI steps of N = 2048; central finite differences on
    9 seeded components (3 each of x, v, m), the differences of L summed with
    compensation.  Positions and velocities use the absolute step 1e-6; masses
    (m = 1/2048) a relative step of 1e-4, because an absolute 1e-6 would be ~2e-3 of m
    and the FD noise of a 1e-9 step (last-bit differences between forward runs,
    amplified over 20 steps) is ~1e-4 of the signal."""
    import math
    from paper_2210_02472_b300.autodiff import fsi_rollout
    c = inputs.plummer(2048, 63)
    h, steps = 1e-3, 20
    with F.Context("fp64") as ctx:
        x = dev(c.pos).requires_grad_(True)
        v = dev(c.vel).requires_grad_(True)
        m = dev(c.mass).requires_grad_(True)
        p, _ = fsi_rollout(ctx, x, v, m, h, steps, ckpt_every=5)
        (p * p).sum().backward()
        grads = [x.grad.cpu().numpy(), v.grad.cpu().numpy(), m.grad.cpu().numpy()]

        def final(px, pv, pm):
            P, V = dev(px), dev(pv)
            F.fsi_step(ctx, P, V, dev(pm), h, nsteps=steps)
            return P.cpu().numpy()

        rng = np.random.default_rng(7)
        for t in range(9):
            which = t % 3
            k, i = int(rng.integers(3)), int(rng.integers(c.n))
            arrs = [c.pos.copy(), c.vel.copy(), c.mass.copy()]
            base = arrs[which]
            idx = (i,) if which == 2 else (k, i)
            step = 1e-4 * base[idx] if which == 2 else 1e-6
            base[idx] += step
            fp = final(*arrs)
            base[idx] -= 2 * step
            fm = final(*arrs)
            fd = math.fsum(((fp * fp) - (fm * fm)).ravel()) / (2 * step)
            an = grads[which][idx]
            tol = 1e-6 * max(1.0, abs(an)) if which < 2 else 1e-5 * abs(an)
            assert abs(fd - an) <= tol, (which, idx, fd, an)


@pytest.mark.parametrize("subset", [False, True])
def test_step_record_matches_step_and_oracle(F, subset):
    """fsi_step_record advances the state exactly like fsi_step (one cycle) and returns
    a(x0), a(x1) and G(x1) of the cycle (x1 after the first kick and drift), against the
    oracle's sums at the oracle's x1."""
    n = 1500
    c = inputs.plummer(n, 64, imf="kroupa")
    h = 1e-3
    P = np.sort(inputs.random_subset(n, 700, 65)).astype(np.int32) if subset else None
    with F.Context("fp64") as ctx:
        idx = None if P is None else dev(P, torch.int32)
        p1, v1 = dev(c.pos), dev(c.vel)
        F.fsi_step(ctx, p1, v1, dev(c.mass), h, nsteps=1, idx=idx)
        p2, v2 = dev(c.pos), dev(c.vel)
        a0, a1, g1 = F.fsi_step_record(ctx, p2, v2, dev(c.mass), h, idx=idx)
        assert F.fsi_sync_status(ctx) == F.FSI_OK
        p1, v1, p2, v2 = (t.cpu().numpy() for t in (p1, v1, p2, v2))
        a0, a1, g1 = (t.cpu().numpy() for t in (a0, a1, g1))
    assert np.abs(p2 - p1).max() <= 1e-14 * np.abs(p1).max()
    assert np.abs(v2 - v1).max() <= 1e-13 * np.abs(v1).max()
    S = np.arange(n) if P is None else P
    ra0 = np.asarray(oracle.acc(c.pos, c.mass, S, S))
    x1 = c.pos.copy()
    x1[:, S] = c.pos[:, S] + 0.5 * h * (c.vel[:, S] + h / 6.0 * ra0)
    ra1 = np.asarray(oracle.acc(x1, c.mass, S, S))
    accg = np.zeros_like(c.pos)
    accg[:, S] = ra1
    rg1 = np.asarray(oracle.grad(x1, c.mass, accg, S, S))
    for got, ref, tol in ((a0, ra0, 1e-12), (a1, ra1, 1e-11), (g1, rg1, 1e-10)):
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max()


def test_step_vjp_rec_matches_recomputing_vjp(F):
    """The adjoint given the recorded intermediates equals the one that recomputes them."""
    n = 2500
    c = inputs.plummer(n, 66, imf="kroupa")
    h = 1e-3
    rng = np.random.default_rng(67)
    gx, gv = rng.normal(size=(3, n)), rng.normal(size=(3, n))
    with F.Context("fp64") as ctx:
        x0, v0, m = dev(c.pos), dev(c.vel), dev(c.mass)
        rec = F.fsi_step_record(ctx, x0.clone(), v0.clone(), m, h)
        r1 = F.fsi_step_vjp(ctx, x0, v0, m, h, dev(gx), dev(gv))
        r2 = F.fsi_step_vjp_rec(ctx, x0, v0, m, h, rec, dev(gx), dev(gv))
        assert F.fsi_sync_status(ctx) == F.FSI_OK
        r1 = [t.cpu().numpy() for t in r1]
        r2 = [t.cpu().numpy() for t in r2]
    for a, b in zip(r2, r1):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
