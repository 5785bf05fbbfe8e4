"""Seeded synthetic star-cluster inputs (Plummer sphere, Kroupa IMF, black holes, ensembles).

This module only draws initial conditions; it holds none of the integrator's arithmetic
(no accelerations, gradients, time steps or energies).  Both the CUDA path and the CPU
oracle are fed from here, so that the two see bit-identical inputs.

Units are Henon N-body units: G = 1, total mass M = 1, and for a Plummer model the scale
radius is a = 3*pi/16 so that the total energy of the model is E = -1/4.

Sampling follows the paper's initial-conditions generator (Appendix A):

* radii by inversion of the Plummer cumulative mass profile M(r) = M r^3 / (r^2 + a^2)^{3/2};
* speeds by von Neumann rejection on the isotropic distribution function f(E) ~ E^{7/2},
  i.e. on q^2 (1 - q^2)^{7/2} with q = v / v_esc(r);
* isotropic directions from two uniform angles on the unit sphere;
* stellar masses from the Kroupa (2001) IMF (slopes 1.3 on [0.08, 0.5] Msun and 2.3 on
  [0.5, 100] Msun; the paper names the IMF but does not print the slopes).

Radii beyond 10 a are re-drawn (a truncation the paper does not state).  The model is
shifted to its centre-of-mass frame.  No virial rescaling is done: the realised energy
differs from -1/4 by sampling noise of order 1/sqrt(N).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

PLUMMER_A = 3.0 * math.pi / 16.0          # Henon-unit Plummer scale radius
KROUPA_BREAK = 0.5                        # Msun
KROUPA_MMIN, KROUPA_MMAX = 0.08, 100.0    # Msun
KROUPA_ALPHA_LO, KROUPA_ALPHA_HI = 1.3, 2.3
SEED_BASE = 20221005


@dataclass
class Cluster:
    """Structure-of-arrays particle set in FP64.

    pos, vel: shape (3, N), rows x, y, z (contiguous per component).
    mass: shape (N,).  is_bh: shape (N,) bool flag for black holes.
    """
    pos: np.ndarray
    vel: np.ndarray
    mass: np.ndarray
    is_bh: np.ndarray

    @property
    def n(self) -> int:
        return int(self.mass.shape[0])


def _unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    """Isotropic unit vectors from cos(theta) ~ U(-1, 1) and phi ~ U(0, 2 pi)."""
    cth = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    return np.stack([sth * np.cos(phi), sth * np.sin(phi), cth])


def _plummer_radii(rng: np.random.Generator, n: int, a: float, rmax: float) -> np.ndarray:
    """Inverse of the Plummer cumulative mass fraction X = r^3/(r^2+a^2)^{3/2}."""
    out = np.empty(n)
    filled = 0
    while filled < n:
        k = n - filled
        x = rng.uniform(0.0, 1.0, k)
        x = x[x > 0.0]
        r = a / np.sqrt(x ** (-2.0 / 3.0) - 1.0)
        r = r[r <= rmax]
        take = min(r.size, n - filled)
        out[filled:filled + take] = r[:take]
        filled += take
    return out


def _plummer_speed_fraction(rng: np.random.Generator, n: int) -> np.ndarray:
    """Rejection sampling of q on [0, 1] with density ~ q^2 (1 - q^2)^{7/2}.

    The density's maximum is below 0.1 (at q^2 = 2/9 it is ~0.092), so the envelope is
    the constant 0.1.
    """
    out = np.empty(n)
    filled = 0
    while filled < n:
        k = max(16, 2 * (n - filled))
        q = rng.uniform(0.0, 1.0, k)
        y = rng.uniform(0.0, 0.1, k)
        acc = q[y < q * q * (1.0 - q * q) ** 3.5]
        take = min(acc.size, n - filled)
        out[filled:filled + take] = acc[:take]
        filled += take
    return out


def _plummer_escape_speed(r: np.ndarray, a: float, mtot: float) -> np.ndarray:
    """v_esc(r) = sqrt(2 |phi(r)|) for the Plummer potential phi = -M / sqrt(r^2 + a^2)."""
    return np.sqrt(2.0 * mtot / np.sqrt(r * r + a * a))


def kroupa_masses(rng: np.random.Generator, n: int) -> np.ndarray:
    """Masses in Msun from the two-segment Kroupa (2001) IMF, inverse-CDF per segment."""
    a1, a2 = KROUPA_ALPHA_LO, KROUPA_ALPHA_HI
    m0, mb, m1 = KROUPA_MMIN, KROUPA_BREAK, KROUPA_MMAX
    # xi(m) = k1 m^-a1 below the break, k2 m^-a2 above, continuous at mb.
    k1 = 1.0
    k2 = k1 * mb ** (a2 - a1)
    w1 = k1 * (mb ** (1 - a1) - m0 ** (1 - a1)) / (1 - a1)
    w2 = k2 * (m1 ** (1 - a2) - mb ** (1 - a2)) / (1 - a2)
    seg = rng.uniform(0.0, 1.0, n) < w1 / (w1 + w2)
    u = rng.uniform(0.0, 1.0, n)

    def inv(lo, hi, alpha, uu):
        p = 1.0 - alpha
        return (lo ** p + uu * (hi ** p - lo ** p)) ** (1.0 / p)

    return np.where(seg, inv(m0, mb, a1, u), inv(mb, m1, a2, u))


def plummer(n: int, seed: int, imf: str = "equal", n_bh: int = 0,
            bh_mass_range=(50.0, 100.0), rmax_over_a: float = 10.0) -> Cluster:
    """A Plummer sphere of n stars (+ n_bh black holes) in Henon units.

    imf: "equal" (all m = 1/N) or "kroupa".  With black holes, their masses are drawn
    uniformly from bh_mass_range in Msun, in the same Msun unit as the stars, and all
    masses are rescaled together so that the total is 1.  The holes are placed uniformly
    inside the radius where the Plummer density falls to half its central value,
    r_c = a (2^{2/5} - 1)^{1/2}, with speeds from the Plummer distribution function at
    their radius.
    """
    rng = np.random.default_rng(np.random.PCG64(seed))
    a = PLUMMER_A
    ntot = n + n_bh
    r = _plummer_radii(rng, n, a, rmax_over_a * a)
    pos = _unit_vectors(rng, n) * r
    q = _plummer_speed_fraction(rng, n)
    vel = _unit_vectors(rng, n) * (q * _plummer_escape_speed(r, a, 1.0))

    if imf == "equal":
        m_msun = np.full(n, 1.0)
    elif imf == "kroupa":
        m_msun = kroupa_masses(rng, n)
    else:
        raise ValueError(f"unknown imf {imf!r}")

    is_bh = np.zeros(ntot, dtype=bool)
    if n_bh > 0:
        rc = a * math.sqrt(2.0 ** 0.4 - 1.0)
        rb = rc * rng.uniform(0.0, 1.0, n_bh) ** (1.0 / 3.0)
        pb = _unit_vectors(rng, n_bh) * rb
        qb = _plummer_speed_fraction(rng, n_bh)
        vb = _unit_vectors(rng, n_bh) * (qb * _plummer_escape_speed(rb, a, 1.0))
        mb = rng.uniform(bh_mass_range[0], bh_mass_range[1], n_bh)
        pos = np.concatenate([pos, pb], axis=1)
        vel = np.concatenate([vel, vb], axis=1)
        m_msun = np.concatenate([m_msun, mb])
        is_bh[n:] = True

    mass = m_msun / m_msun.sum()
    com = (pos * mass).sum(axis=1, keepdims=True)
    vcom = (vel * mass).sum(axis=1, keepdims=True)
    pos = np.ascontiguousarray(pos - com)
    vel = np.ascontiguousarray(vel - vcom)
    return Cluster(pos=pos, vel=vel, mass=np.ascontiguousarray(mass), is_bh=is_bh)


def ensemble_sizes(k: int, nmin: int, nmax: int, seed: int) -> np.ndarray:
    """Cluster sizes log-uniform in [nmin, nmax] (integers, inclusive)."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    ln = rng.uniform(math.log(nmin), math.log(nmax + 1), k)
    return np.clip(np.floor(np.exp(ln)).astype(np.int64), nmin, nmax)


def ensemble(k: int, nmin: int, nmax: int, seed: int, imf: str = "kroupa"):
    """k independent Plummer clusters, each in its own Henon units, concatenated.

    Returns (Cluster of the concatenation, offsets[k+1]).
    """
    sizes = ensemble_sizes(k, nmin, nmax, seed)
    parts = [plummer(int(nk), seed * 7919 + 1 + c, imf=imf) for c, nk in enumerate(sizes)]
    offsets = np.zeros(k + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    cat = Cluster(
        pos=np.ascontiguousarray(np.concatenate([p.pos for p in parts], axis=1)),
        vel=np.ascontiguousarray(np.concatenate([p.vel for p in parts], axis=1)),
        mass=np.concatenate([p.mass for p in parts]),
        is_bh=np.concatenate([p.is_bh for p in parts]),
    )
    return cat, offsets


def random_subset(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct indices of [0, n), sorted, as int32."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int32)


def random_field(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """A seeded (3, n) FP64 vector field with normal components (stand-in accelerations)."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    return np.ascontiguousarray(rng.normal(0.0, scale, (3, n)))


# Named workloads (sizes and seeds) used by the tests and the benchmark.
def workload(name: str) -> Cluster:
    if name == "plummer1k":        # 1024 equal-mass stars
        return plummer(1024, SEED_BASE + 1, imf="equal")
    if name == "kroupa64k":        # 65536 stars, Kroupa IMF
        return plummer(65536, SEED_BASE + 2, imf="kroupa")
    if name == "kroupa1m_bh16":    # 2^20 stars, Kroupa IMF, plus 16 black holes
        return plummer(1 << 20, SEED_BASE + 3, imf="kroupa", n_bh=16)
    if name == "plummer16k":       # 16384 equal-mass stars
        return plummer(16384, SEED_BASE + 4, imf="equal")
    if name == "plummer161k":      # 161000 equal-mass stars (the softened long-run cluster)
        return plummer(161000, SEED_BASE + 6, imf="equal")
    raise KeyError(name)
