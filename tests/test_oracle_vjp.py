"""Pins of the oracle's hand-derived adjoint (VJP) of the FSI cycle.

Independent references: central finite differences of the (separately pinned) forward
oracle, and reverse-mode automatic differentiation (torch, float64, CPU) of a forward FSI
step restated here from the paper's equations (Sect. 2.1), itself checked against the
forward oracle first.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2210_02472_b300 import inputs


def rand_like(shape, seed):
    return np.random.default_rng(seed).normal(size=shape)


@pytest.mark.parametrize("eps2", [0.0, 1e-3])
def test_vjp_acc_matches_finite_differences(eps2):
    c = inputs.plummer(24, 51, imf="kroupa")
    u = rand_like((3, c.n), 1)
    xb, mb = oracle.vjp_acc(c.pos, c.mass, u, eps2=eps2)
    dx = rand_like((3, c.n), 2)
    dm = rand_like(c.n, 3) * c.mass
    e = 1e-6

    def L(p, m):
        return float((u * oracle.acc(p, m, eps2=eps2)).sum())

    fd_x = (L(c.pos + e * dx, c.mass) - L(c.pos - e * dx, c.mass)) / (2 * e)
    fd_m = (L(c.pos, c.mass + e * dm) - L(c.pos, c.mass - e * dm)) / (2 * e)
    assert abs(fd_x - (xb * dx).sum()) < 1e-7 * abs(fd_x) + 1e-9
    assert abs(fd_m - (mb * dm).sum()) < 1e-7 * abs(fd_m) + 1e-9


@pytest.mark.parametrize("eps2", [0.0, 1e-3])
def test_vjp_grad_matches_finite_differences(eps2):
    """VJP of G(r, m; a) with the accelerations held fixed."""
    c = inputs.plummer(20, 52, imf="kroupa")
    acc = rand_like((3, c.n), 4)
    w = rand_like((3, c.n), 5)
    xb, mb = oracle.vjp_grad(c.pos, c.mass, acc, w, eps2=eps2)
    dx = rand_like((3, c.n), 6)
    dm = rand_like(c.n, 7) * c.mass
    e = 1e-6

    def L(p, m):
        return float((w * oracle.grad(p, m, acc, eps2=eps2)).sum())

    fd_x = (L(c.pos + e * dx, c.mass) - L(c.pos - e * dx, c.mass)) / (2 * e)
    fd_m = (L(c.pos, c.mass + e * dm) - L(c.pos, c.mass - e * dm)) / (2 * e)
    assert abs(fd_x - (xb * dx).sum()) < 1e-6 * abs(fd_x) + 1e-8
    assert abs(fd_m - (mb * dm).sum()) < 1e-6 * abs(fd_m) + 1e-8


def step_pair(c, h, gx, gv, dx, dv, dm, e):
    def L(p, v, m):
        p1, v1 = oracle.fsi_step(p, v, m, h)
        return float((gx * p1).sum() + (gv * v1).sum())
    return (L(c.pos + e * dx, c.vel + e * dv, c.mass + e * dm)
            - L(c.pos - e * dx, c.vel - e * dv, c.mass - e * dm)) / (2 * e)


def test_step_vjp_matches_finite_differences():
    c = inputs.plummer(32, 53, imf="kroupa")
    h = 2e-3
    gx, gv = rand_like((3, c.n), 8), rand_like((3, c.n), 9)
    ix, iv, im = oracle.fsi_step_vjp(c.pos, c.vel, c.mass, h, gx, gv)
    for seed in range(3):
        dx, dv = rand_like((3, c.n), 10 + seed), rand_like((3, c.n), 20 + seed)
        dm = rand_like(c.n, 30 + seed) * c.mass
        fd = step_pair(c, h, gx, gv, dx, dv, dm, 1e-6)
        an = (ix * dx).sum() + (iv * dv).sum() + (im * dm).sum()
        assert abs(fd - an) < 1e-7 * abs(fd), (fd, an)


# --- independent forward restatement in torch (Sect. 2.1), differentiated by autograd
def torch_acc(x, m, eps2=0.0):
    d = x[:, None, :] - x[:, :, None]            # d[:, i, j] = x_j - x_i
    r2 = (d * d).sum(0) + eps2
    n = x.shape[1]
    eye = torch.eye(n, dtype=torch.bool)
    inv3 = torch.where(eye, torch.zeros_like(r2), r2.clamp_min(1e-300) ** -1.5)
    return (d * (m[None, None, :] * inv3)).sum(2)


def torch_grad(x, m, a, eps2=0.0):
    d = x[:, None, :] - x[:, :, None]
    r2 = (d * d).sum(0) + eps2
    n = x.shape[1]
    eye = torch.eye(n, dtype=torch.bool)
    r2s = torch.where(eye, torch.ones_like(r2), r2)
    b = a[:, None, :] - a[:, :, None]            # b[:, i, j] = a_j - a_i
    ab = (b * d).sum(0)
    term = (r2s * b - 3.0 * ab * d) * (m[None, None, :] / r2s ** 2.5)
    term = torch.where(eye[None], torch.zeros_like(term), term)
    return term.sum(2)


def torch_step(x, v, m, h):
    v = v + h / 6 * torch_acc(x, m)
    x = x + h / 2 * v
    a = torch_acc(x, m)
    v = v + 2 * h / 3 * (a + h * h / 24 * torch_grad(x, m, a))
    x = x + h / 2 * v
    v = v + h / 6 * torch_acc(x, m)
    return x, v


def test_step_vjp_matches_autograd_of_restated_forward():
    c = inputs.plummer(12, 54, imf="kroupa")
    h = 5e-3
    x = torch.tensor(c.pos, requires_grad=True)
    v = torch.tensor(c.vel, requires_grad=True)
    m = torch.tensor(c.mass, requires_grad=True)
    x1, v1 = torch_step(x, v, m, h)
    rp, rv = oracle.fsi_step(c.pos, c.vel, c.mass, h)
    assert np.abs(x1.detach().numpy() - rp).max() < 1e-13
    assert np.abs(v1.detach().numpy() - rv).max() < 1e-12
    gx, gv = rand_like((3, c.n), 11), rand_like((3, c.n), 12)
    (x1 * torch.tensor(gx)).sum().add((v1 * torch.tensor(gv)).sum()).backward()
    ix, iv, im = oracle.fsi_step_vjp(c.pos, c.vel, c.mass, h, gx, gv)
    assert np.abs(ix - x.grad.numpy()).max() < 1e-10 * np.abs(ix).max()
    assert np.abs(iv - v.grad.numpy()).max() < 1e-12 * np.abs(iv).max()
    assert np.abs(im - m.grad.numpy()).max() < 1e-10 * np.abs(im).max()


def test_step_vjp_subset_passes_others_through():
    c = inputs.plummer(20, 55)
    P = np.arange(0, 20, 2, dtype=np.int32)
    gx, gv = rand_like((3, c.n), 13), rand_like((3, c.n), 14)
    ix, iv, im = oracle.fsi_step_vjp(c.pos, c.vel, c.mass, 1e-3, gx, gv, P=P)
    others = np.arange(1, 20, 2)
    assert np.array_equal(ix[:, others], gx[:, others])
    assert np.array_equal(iv[:, others], gv[:, others])
    assert np.all(im[others] == 0)
