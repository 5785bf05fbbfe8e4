"""i-sharded pair passes, FSI cycles and HHS intervals over several ranks (one process per
GPU).

Direct summation shards along the receivers: every rank holds the replicated positions
and masses of the whole set (and, for the gradient pass, the accelerations of the whole
splitting term), and computes the pair sums of a contiguous slice of the active list
against all sources.  The data exchanged between ranks is what the next pass needs:

  * after every drift, an all-gather of the moved particles' positions (24 B per particle
    of the active list);
  * between the acceleration and the gradient pass, an all-gather of the accelerations of
    the splitting term (24 B per particle of A, and of B for an inter-level term), since
    the gradient sum of Sect. 2.1 (Eq. new-grad-acc) needs a_j of every source j;
  * for active sets too small to give every rank receivers (fewer than `min_rows` per
    rank), the sources are split instead and the partial acceleration and gradient sums
    are all-reduced (48 B per active particle).

With `pairs=True` (and a compute that has the share form) the same-set passes of the pair
sums and of FSI cycles are split by pairs instead of rows: every rank evaluates its share
of the set's unordered pairs for both particles of each (Newton's third law: half the pair
evaluations of a row split), the shares are all-reduced (24 B per particle and pass), and
every rank kicks and drifts the whole set with the same sums, so the replicated positions
stay identical without an all-gather.

An HHS interval shards every level's active list the same way: the inter-level kicks split
the rows of S and F, and FSI(S) is a sharded FSI cycle of S.

The paper runs its direct-summation loops on several GPUs with MPI (Sect. 4.1); here the
collectives are torch.distributed's (NCCL between GPUs: every operand lands in the
receiving GPU's own memory before a kernel reads it).  The exchange layer only moves
data: every pair sum, kick and drift is done by the shard compute, which for the product
is libfsi on the rank's own GPU (LibfsiCompute); the tests plug the CPU oracle in
instead to check the exchange against one-rank results on gloo ranks.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import torch


def slice_bounds(n: int, world: int, rank: int):
    """Contiguous slice [lo, hi) of an n-entry list owned by `rank`: the first n % world
    ranks take one entry more."""
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


class LibfsiCompute:
    """Shard compute on the rank's GPU through libfsi's C ABI (a context per rank).
    Index lists are int32 CUDA tensors of global ids."""

    def __init__(self, ctx):
        from . import fsi
        self.F = fsi
        self.ctx = ctx

    def accel(self, pos, mass, A, B, eps2):
        return self.F.fsi_accel(self.ctx, pos, mass, A, B, eps2=eps2)

    def grad(self, pos, mass, accg, A, B, eps2):
        return self.F.fsi_grad(self.ctx, pos, mass, accg, A, B, eps2=eps2)

    def accel_part(self, pos, mass, A, part, nparts, eps2):
        return self.F.fsi_accel_part(self.ctx, pos, mass, part, nparts, A, eps2=eps2)

    def grad_part(self, pos, mass, accg, A, part, nparts, eps2):
        return self.F.fsi_grad_part(self.ctx, pos, mass, accg, part, nparts, A, eps2=eps2)

    def pn_accel(self, pos, vel, mass, is_bh, c, A, B):
        return self.F.fsi_pn_accel(self.ctx, pos, vel, mass, is_bh, c, A, B)

    def kick_drift(self, pos, vel, acc, idx, c_kick, c_drift):
        self.F.fsi_kick_drift(self.ctx, pos, vel, acc, c_kick, c_drift, idx=idx)

    def timesteps(self, pos, vel, mass, P, eps2):
        """Time steps of the set P against itself with the context's criteria; eps2 must be
        the context's (the time-step call takes it from there)."""
        self._check_eps2(eps2)
        return self.F.fsi_timesteps(self.ctx, pos, vel, mass, P)

    def timesteps_rows(self, pos, vel, mass, P, lo, hi, eps2):
        """Time steps of P[lo:hi] against the whole set P, or None when the context's
        gradient criteria are on (they need the whole set's accelerations)."""
        self._check_eps2(eps2)
        if self.ctx.params.eta_grad > 0.0 or self.ctx.params.eta_va > 0.0:
            return None
        return self.F.fsi_timesteps_sub(self.ctx, pos, vel, mass, P, lo, hi)

    def _check_eps2(self, eps2):
        if float(self.ctx.params.eps2) != float(eps2):
            raise ValueError("timesteps: eps2 differs from the context's fsi_params.eps2")

    def status(self):
        return self.F.fsi_sync_status(self.ctx)


class Exchange:
    """Collectives of the sharded passes over a torch.distributed process group (None:
    a single rank).  With a CPU backend (gloo) and device tensors, operands are staged
    through host memory."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist if dist.is_available() and dist.is_initialized() else None
        self.group = group
        self.world = self.dist.get_world_size(group) if self.dist else 1
        self.rank = self.dist.get_rank(group) if self.dist else 0
        self.cpu_backend = bool(self.dist) and self.dist.get_backend(group) == "gloo"

    def _stage(self, t):
        return t.cpu() if (self.cpu_backend and t.is_cuda) else t

    def all_gather_cols(self, local: torch.Tensor, n: int) -> torch.Tensor:
        """Concatenate the ranks' (rows, n_r) column slices (slice_bounds order) into
        (rows, n)."""
        if self.dist is None:
            return local
        q = -(-n // self.world)
        rows = local.shape[0]
        buf = torch.zeros((rows, q), dtype=local.dtype, device=local.device)
        buf[:, :local.shape[1]] = local
        sb = self._stage(buf.contiguous())
        parts = [torch.empty_like(sb) for _ in range(self.world)]
        self.dist.all_gather(parts, sb, group=self.group)
        cols = []
        for r, p in enumerate(parts):
            lo, hi = slice_bounds(n, self.world, r)
            cols.append(p[:, :hi - lo])
        return torch.cat(cols, dim=1).to(local.device)

    def all_reduce_sum(self, t: torch.Tensor) -> torch.Tensor:
        if self.dist is None:
            return t
        st = self._stage(t.contiguous())
        self.dist.all_reduce(st, op=self.dist.ReduceOp.SUM, group=self.group)
        return st.to(t.device)


@dataclass
class ShardPlan:
    """Which receivers (or, for small active sets, which sources) a rank takes."""
    mode: str                  # "rows": a slice of A against all of B; "sources": all of A
    lo: int                    # against a slice of B
    hi: int


def plan(nA: int, nB: int, ex: Exchange, min_rows: int) -> ShardPlan:
    if ex.world > 1 and nA < min_rows * ex.world and nB >= ex.world:
        lo, hi = slice_bounds(nB, ex.world, ex.rank)
        return ShardPlan("sources", lo, hi)
    lo, hi = slice_bounds(nA, ex.world, ex.rank)
    return ShardPlan("rows", lo, hi)


def _ids(n: int, idx: Optional[torch.Tensor], device) -> torch.Tensor:
    return idx if idx is not None else torch.arange(n, dtype=torch.int32, device=device)


class ShardedFSI:
    """The sharded hot path: pair sums of one splitting term (fsi_accel_grad semantics),
    FSI cycles of a set (fsi_step semantics) and HHS intervals (fsi_hhs_interval
    semantics), with every rank ending with the same results.  `compute` does all
    arithmetic; `ex` moves data between ranks."""

    def __init__(self, compute, ex: Optional[Exchange] = None, min_rows: int = 1024,
                 pairs: bool = False):
        self.c = compute
        self.ex = ex or Exchange()
        self.min_rows = int(min_rows)
        self.pairs = bool(pairs) and hasattr(compute, "accel_part") and hasattr(compute, "grad_part")

    def _split_pairs(self) -> bool:
        return self.pairs and self.ex.world > 1

    def _acc_share(self, pos, mass, P, eps2):
        """acc(P <- P) on every rank: this rank's share of the pairs, all-reduced."""
        return self.ex.all_reduce_sum(self.c.accel_part(pos, mass, P, self.ex.rank, self.ex.world, eps2))

    def _grad_share(self, pos, mass, accg, P, eps2):
        return self.ex.all_reduce_sum(self.c.grad_part(pos, mass, accg, P, self.ex.rank,
                                                       self.ex.world, eps2))

    # -------------------------------------------------------------- pair sums
    def _acc(self, pos, mass, A, B, eps2, p: ShardPlan):
        if p.mode == "rows":
            a = self.c.accel(pos, mass, A[p.lo:p.hi], B, eps2)
            return self.ex.all_gather_cols(a, A.numel())
        return self.ex.all_reduce_sum(self.c.accel(pos, mass, A, B[p.lo:p.hi], eps2))

    def _grad(self, pos, mass, accg, A, B, eps2, p: ShardPlan):
        if p.mode == "rows":
            g = self.c.grad(pos, mass, accg, A[p.lo:p.hi], B, eps2)
            return self.ex.all_gather_cols(g, A.numel())
        return self.ex.all_reduce_sum(self.c.grad(pos, mass, accg, A, B[p.lo:p.hi], eps2))

    def accel_grad(self, pos, mass, A=None, B=None, eps2: float = 0.0):
        """acc(A <- B) and G(A <- B) of one splitting term (Sect. 2.1 / 2.2), both (3, nA)
        on every rank: A and B the same list (or both None) -- the a_j inside G are
        acc(A <- A); A and B disjoint -- a_i = acc(A <- B), a_j = acc(B <- A) (the
        inter-level term).  As for fsi_accel_grad, other overlaps are not a splitting
        term."""
        N = mass.numel()
        same = (A is None and B is None) or (A is not None and A is B)
        A = _ids(N, A, pos.device)
        B = A if same else _ids(N, B, pos.device)
        if same and self._split_pairs():
            a = self._acc_share(pos, mass, A, eps2)
            accg = torch.zeros((3, N), dtype=pos.dtype, device=pos.device)
            accg[:, A.long()] = a
            return a, self._grad_share(pos, mass, accg, A, eps2)
        pa = plan(A.numel(), B.numel(), self.ex, self.min_rows)
        a = self._acc(pos, mass, A, B, eps2, pa)
        accg = torch.zeros((3, N), dtype=pos.dtype, device=pos.device)
        accg[:, A.long()] = a
        if not same:
            pb = plan(B.numel(), A.numel(), self.ex, self.min_rows)
            accg[:, B.long()] = self._acc(pos, mass, B, A, eps2, pb)
        g = self._grad(pos, mass, accg, A, B, eps2, pa)
        return a, g

    # -------------------------------------------------------------- FSI cycles
    def _sync_cols(self, x, idx, lo, hi, n):
        """Every rank's slice idx[lo:hi] of the (3, N) array x, gathered into x[:, idx]."""
        if self.ex.dist is None:
            return
        mine = x[:, idx[lo:hi].long()]
        x[:, idx.long()] = self.ex.all_gather_cols(mine, n)

    def step(self, pos, vel, mass, h: float, nsteps: int = 1, idx=None, eps2: float = 0.0,
             c: float = 0.0, is_bh=None):
        """nsteps FSI cycles (Sect. 2.1, Eq. fsi-cycle) of the set idx (None: all N) on
        itself, in place on the replicated pos / vel: kick h/6, drift h/2, kick 2h/3 with
        a + h^2/24 G, drift h/2, kick h/6, consecutive cycles sharing the closing and
        opening acceleration (a kick of h/3); with c > 0 PN1.0 half-kicks of h/2 wrap every
        cycle (Sect. 3.9; velocities from the start of each half-kick).  Each rank kicks
        and drifts its slice of the set; positions (after drifts), the accelerations of the
        gradient pass and, around PN kicks and at the end, velocities are all-gathered."""
        N = mass.numel()
        P = _ids(N, idx, pos.device)
        n = P.numel()
        if n == 0 or nsteps <= 0:
            return
        if self._split_pairs():
            return self._step_pairs(pos, vel, mass, h, nsteps, P, eps2, c, is_bh)
        lo, hi = slice_bounds(n, self.ex.world, self.ex.rank)
        Pr = P[lo:hi]
        pn = c > 0.0

        def acc_mine():
            return self.c.accel(pos, mass, Pr, P, eps2)

        def pn_kick():
            self._sync_cols(vel, P, lo, hi, n)
            apn = self.c.pn_accel(pos, vel, mass, is_bh, c, Pr, P)
            self.c.kick_drift(pos, vel, apn, Pr, 0.5 * h, 0.0)

        if pn:
            pn_kick()
        a = acc_mine()
        self.c.kick_drift(pos, vel, a, Pr, h / 6.0, 0.5 * h)
        for k in range(nsteps):
            last = k == nsteps - 1
            self._sync_cols(pos, P, lo, hi, n)
            a = acc_mine()
            accg = torch.zeros((3, N), dtype=pos.dtype, device=pos.device)
            accg[:, P.long()] = self.ex.all_gather_cols(a, n)
            g = self.c.grad(pos, mass, accg, Pr, P, eps2)
            self.c.kick_drift(pos, vel, a, Pr, 2.0 * h / 3.0, 0.0)
            self.c.kick_drift(pos, vel, g, Pr, (2.0 * h / 3.0) * (h * h / 24.0), 0.5 * h)
            self._sync_cols(pos, P, lo, hi, n)
            a = acc_mine()
            if not pn and not last:
                self.c.kick_drift(pos, vel, a, Pr, h / 3.0, 0.5 * h)
                continue
            self.c.kick_drift(pos, vel, a, Pr, h / 6.0, 0.0)
            if pn:
                pn_kick()
            if not last:
                # the next cycle's opening kick reuses this acceleration (no drift between)
                pn_kick()
                self.c.kick_drift(pos, vel, a, Pr, h / 6.0, 0.5 * h)
        self._sync_cols(vel, P, lo, hi, n)

    def _step_pairs(self, pos, vel, mass, h, nsteps, P, eps2, c, is_bh):
        """step() with its same-set passes split by pairs: every rank gets the set's full
        sums from the all-reduced shares and kicks and drifts all of P itself (the PN1.0
        terms, pairs with a black hole, are evaluated whole on every rank)."""
        N = mass.numel()
        pn = c > 0.0

        def pn_kick():
            apn = self.c.pn_accel(pos, vel, mass, is_bh, c, P, P)
            self.c.kick_drift(pos, vel, apn, P, 0.5 * h, 0.0)

        if pn:
            pn_kick()
        a = self._acc_share(pos, mass, P, eps2)
        self.c.kick_drift(pos, vel, a, P, h / 6.0, 0.5 * h)
        for k in range(nsteps):
            last = k == nsteps - 1
            a = self._acc_share(pos, mass, P, eps2)
            accg = torch.zeros((3, N), dtype=pos.dtype, device=pos.device)
            accg[:, P.long()] = a
            g = self._grad_share(pos, mass, accg, P, eps2)
            self.c.kick_drift(pos, vel, a, P, 2.0 * h / 3.0, 0.0)
            self.c.kick_drift(pos, vel, g, P, (2.0 * h / 3.0) * (h * h / 24.0), 0.5 * h)
            a = self._acc_share(pos, mass, P, eps2)
            if not pn and not last:
                self.c.kick_drift(pos, vel, a, P, h / 3.0, 0.5 * h)
                continue
            self.c.kick_drift(pos, vel, a, P, h / 6.0, 0.0)
            if pn:
                pn_kick()
            if not last:
                pn_kick()
                self.c.kick_drift(pos, vel, a, P, h / 6.0, 0.5 * h)

    # -------------------------------------------------------------- HHS intervals
    def hhs_interval(self, pos, vel, mass, tau: float, eps2: float = 0.0, c: float = 0.0,
                     is_bh=None, max_level: int = 40):
        """One HHS interval of length tau over all N particles (Sect. 2.2, Eq.
        hhsfsi-cycle), in place on the replicated pos / vel, with every level's active list
        sharded over the ranks: per level visit the time steps of the level set (each rank
        those of its slice against the whole set, all-gathered; in full on every rank when
        the compute has no slice form or declines it, as libfsi does with the gradient
        criteria on), the split S = {eps >= tau}, F = {eps < tau} with the level-step rule (level 0
        records its steps, deeper levels take the min with them; at max_level every
        particle stays in S), then U_SF(tau/6) FSI(S, tau/2) HHS(F, tau/2) U~_SF(2 tau/3)
        HHS(F, tau/2) FSI(S, tau/2) U_SF(tau/6), with PN1.0 S-F kicks of tau/2 around the
        opening and closing U_SF when c > 0 (Sect. 3.9).  The inter-level kicks split S and
        F into row slices, all-gather their accelerations (and, for U~_SF, the gradient
        sums) and kick on every rank; FSI(S) is `step`.  Returns (level_counts,
        maxlevel_hit); the compute's time-step criteria must use the same eps2."""
        N = mass.numel()
        self._hhs_step0 = torch.zeros(N, dtype=pos.dtype, device=pos.device)
        counts = [0] * (max_level + 1)
        hit = [False]
        P = torch.arange(N, dtype=torch.int32, device=pos.device)
        self._hhs(pos, vel, mass, P, float(tau), 0, float(eps2), float(c), is_bh,
                  int(max_level), counts, hit)
        while len(counts) > 1 and counts[-1] == 0:
            counts.pop()
        return counts, hit[0]

    def _hhs(self, pos, vel, mass, P, tau, level, eps2, c, is_bh, max_level, counts, hit):
        """HHS(P, tau) at `level` (see hhs_interval)."""
        n = P.numel()
        if n == 0:
            return
        st = None
        rows = getattr(self.c, "timesteps_rows", None)
        if rows is not None and self.ex.world > 1:
            # each rank the steps of its slice, all-gathered (the same choice on every
            # rank: it depends only on the compute's parameters)
            lo, hi = slice_bounds(n, self.ex.world, self.ex.rank)
            mine = rows(pos, vel, mass, P, lo, hi, eps2)
            if mine is not None:
                st = self.ex.all_gather_cols(mine.to(pos.dtype).reshape(1, -1), n)[0]
        if st is None:
            st = self.c.timesteps(pos, vel, mass, P, eps2).to(pos.dtype)
        Pl = P.long()
        if level == 0:
            self._hhs_step0[Pl] = st
        else:
            st = torch.minimum(st, self._hhs_step0[Pl])
        fast = st < tau
        if level >= max_level:
            if bool(fast.any()):
                hit[0] = True
            fast = torch.zeros_like(fast)
        S, F = P[~fast], P[fast]                     # stable: list order kept
        counts[level] += S.numel()
        cross = S.numel() > 0 and F.numel() > 0
        pn = c > 0.0
        if cross and pn:
            self._pn_cross(pos, vel, mass, S, F, 0.5 * tau, c, is_bh)
        if cross:
            self._cross(pos, vel, mass, S, F, tau / 6.0, eps2)
        if S.numel():
            self.step(pos, vel, mass, 0.5 * tau, 1, idx=S, eps2=eps2, c=c, is_bh=is_bh)
        if F.numel():
            self._hhs(pos, vel, mass, F, 0.5 * tau, level + 1, eps2, c, is_bh, max_level, counts, hit)
        if cross:
            self._cross(pos, vel, mass, S, F, 2.0 * tau / 3.0, eps2, grad_eps=tau)
        if F.numel():
            self._hhs(pos, vel, mass, F, 0.5 * tau, level + 1, eps2, c, is_bh, max_level, counts, hit)
        if S.numel():
            self.step(pos, vel, mass, 0.5 * tau, 1, idx=S, eps2=eps2, c=c, is_bh=is_bh)
        if cross:
            self._cross(pos, vel, mass, S, F, tau / 6.0, eps2)
            if pn:
                self._pn_cross(pos, vel, mass, S, F, 0.5 * tau, c, is_bh)

    def _cross(self, pos, vel, mass, S, F, w, eps2, grad_eps=None):
        """Inter-level kick of S and F (Sect. 2.2): v_S += w acc(S <- F), v_F += w acc(F <- S);
        with grad_eps, the accelerations a + (grad_eps^2 / 24) G of the same inter-level
        term.  Rows of S and F are split over the ranks; the gathered sums are applied on
        every rank."""
        N = mass.numel()
        nS, nF = S.numel(), F.numel()
        pS = plan(nS, nF, self.ex, self.min_rows)
        pF = plan(nF, nS, self.ex, self.min_rows)
        aS = self._acc(pos, mass, S, F, eps2, pS)
        aF = self._acc(pos, mass, F, S, eps2, pF)
        if grad_eps is not None:
            accg = torch.zeros((3, N), dtype=pos.dtype, device=pos.device)
            accg[:, S.long()] = aS
            accg[:, F.long()] = aF
            cg = grad_eps * grad_eps / 24.0
            aS = aS + cg * self._grad(pos, mass, accg, S, F, eps2, pS)
            aF = aF + cg * self._grad(pos, mass, accg, F, S, eps2, pF)
        self.c.kick_drift(pos, vel, aS, S, w, 0.0)
        self.c.kick_drift(pos, vel, aF, F, w, 0.0)

    def _pn_cross(self, pos, vel, mass, S, F, w, c, is_bh):
        """PN1.0 kick of the S-F pairs (Sect. 3.9), both directions, from the velocities at
        the start of the kick: rows split over the ranks, the sums gathered and applied on
        every rank."""
        nS, nF = S.numel(), F.numel()
        lo, hi = slice_bounds(nS, self.ex.world, self.ex.rank)
        pS = self.ex.all_gather_cols(self.c.pn_accel(pos, vel, mass, is_bh, c, S[lo:hi], F), nS)
        lo, hi = slice_bounds(nF, self.ex.world, self.ex.rank)
        pF = self.ex.all_gather_cols(self.c.pn_accel(pos, vel, mass, is_bh, c, F[lo:hi], S), nF)
        self.c.kick_drift(pos, vel, pS, S, w, 0.0)
        self.c.kick_drift(pos, vel, pF, F, w, 0.0)
