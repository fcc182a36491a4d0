"""The solve phase split over several ranks (one GPU each): decomposition
and communication schedule.

The method's subdomains are independent units for the local solves, the
restriction and the prolongation (Section 3.2: the fine-level term and the
blocks of R_0^T live on one subdomain each), so the path shards by
contiguous ranges of subdomains.  In the subdomain-major order of
Section 3.1 such a range is a contiguous block of rows, and its coarse
unknowns (the m_i modes of its subdomains, Section 3.2) are a contiguous
block of the coarse vector.  One CG iteration then needs:

* one halo exchange before the SpMV: each rank receives the entries of the
  direction p at the columns its rows reference outside its own block
  (point-to-point, only between ranks whose blocks are coupled);
* one all-reduce of p.q after the SpMV (the step length);
* one all-gather of the restricted residual r_c = R_0 r (every rank's
  block of it), after which every rank runs the same coarse substitutions
  on the replicated coarse factor and keeps its own block of e_c;
* one all-reduce of the fused dots r.r, r.z and z.q after the
  preconditioner (convergence test and the next direction's beta).

Everything else is local to a rank.  This module holds the host side: the
plan (ranges, ghost lists, send and receive lists, the rank's rows of A
with columns renumbered into owned-then-ghost order) and the iteration
driver, which does no arithmetic of its own: every vector operation goes
through a per-rank operator object and every exchange through a
communicator over ``torch.distributed``.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Protocol

import numpy as np


# ---------------------------------------------------------------------------
# plan
# ---------------------------------------------------------------------------

@dataclass
class RankPlan:
    rank: int
    sub_lo: int                  # first subdomain of this rank
    sub_hi: int                  # one past the last
    row_lo: int                  # first internal row (subdomain-major order)
    row_hi: int
    coarse_lo: int               # first coarse unknown (paper order)
    coarse_hi: int
    ghost: np.ndarray            # internal rows of other ranks this rank's rows reference (ascending)
    recv: dict = field(default_factory=dict)   # peer -> positions in `ghost` received from it
    send: dict = field(default_factory=dict)   # peer -> owned rows (local index) sent to it
    rowptr: Optional[np.ndarray] = None        # owned rows of A, internal order,
    colind: Optional[np.ndarray] = None        # columns: local owned index, then n_owned + ghost position
    vals: Optional[np.ndarray] = None
    entry: Optional[np.ndarray] = None         # caller CSR entry of each of those entries

    @property
    def n_owned(self) -> int:
        return self.row_hi - self.row_lo


@dataclass
class ShardPlan:
    world: int
    n: int
    nparts: int
    perm: np.ndarray             # internal position -> caller dof
    sub_ptr: np.ndarray          # internal row range of each subdomain
    coarse_ptr: np.ndarray       # coarse range of each subdomain (paper order)
    ranks: List[RankPlan]


def _subdomain_order(part: np.ndarray, nparts: int):
    """Subdomain-major order (Section 3.1): subdomain by subdomain, each in
    ascending caller index."""
    order = np.argsort(part, kind="stable")
    counts = np.bincount(part, minlength=nparts)
    sub_ptr = np.zeros(nparts + 1, dtype=np.int64)
    sub_ptr[1:] = np.cumsum(counts)
    return order.astype(np.int64), sub_ptr


def balanced_ranges(sub_ptr: np.ndarray, world: int) -> np.ndarray:
    """First subdomain of each rank (world + 1 entries): contiguous ranges
    whose row counts are as even as whole subdomains allow, every rank
    holding at least one subdomain."""
    nparts = len(sub_ptr) - 1
    if not 1 <= world <= nparts:
        raise ValueError(f"world size {world} must be between 1 and the {nparts} subdomains")
    n = int(sub_ptr[-1])
    lo = [0]
    for r in range(1, world):
        target = n * r / world
        k = int(np.searchsorted(sub_ptr, target))           # first boundary at or past the target
        if k > 0 and abs(sub_ptr[k - 1] - target) <= abs(sub_ptr[min(k, nparts)] - target):
            k -= 1
        k = max(k, lo[-1] + 1)                              # at least one subdomain each
        k = min(k, nparts - (world - r))
        lo.append(k)
    lo.append(nparts)
    return np.asarray(lo, dtype=np.int64)


def make_plan(rowptr, colind, vals, part, nparts: int, m_i, world: int) -> ShardPlan:
    """Split one system over `world` ranks by contiguous subdomain ranges."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    colind = np.asarray(colind, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    part = np.asarray(part, dtype=np.int64)
    n = len(rowptr) - 1
    perm, sub_ptr = _subdomain_order(part, nparts)
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    m_i = np.asarray(m_i, dtype=np.int64)
    coarse_ptr = np.zeros(nparts + 1, dtype=np.int64)
    coarse_ptr[1:] = np.cumsum(m_i)
    slo = balanced_ranges(sub_ptr, world)
    row_lo = sub_ptr[slo]
    owner = np.searchsorted(row_lo, np.arange(n), side="right") - 1   # internal row -> rank
    ranks = []
    for r in range(world):
        a, b = int(row_lo[r]), int(row_lo[r + 1])
        rows = perm[a:b]                                   # caller dofs of the owned rows, in order
        starts, ends = rowptr[rows], rowptr[rows + 1]
        cnt = ends - starts
        src = np.concatenate([np.arange(s, e) for s, e in zip(starts, ends)]) if len(rows) else \
            np.zeros(0, dtype=np.int64)
        cols_int = iperm[colind[src]]                      # internal column indices
        ghost = np.unique(cols_int[(cols_int < a) | (cols_int >= b)])
        local = np.where((cols_int >= a) & (cols_int < b), cols_int - a,
                         (b - a) + np.searchsorted(ghost, cols_int))
        lrp = np.zeros(len(rows) + 1, dtype=np.int64)
        lrp[1:] = np.cumsum(cnt)
        rp = RankPlan(rank=r, sub_lo=int(slo[r]), sub_hi=int(slo[r + 1]), row_lo=a, row_hi=b,
                      coarse_lo=int(coarse_ptr[slo[r]]), coarse_hi=int(coarse_ptr[slo[r + 1]]),
                      ghost=ghost, rowptr=lrp, colind=local, vals=vals[src], entry=src)
        gown = owner[ghost]
        for q in np.unique(gown):
            rp.recv[int(q)] = np.flatnonzero(gown == q)
        ranks.append(rp)
    for r, rp in enumerate(ranks):                         # sends mirror the peers' receives
        for q, pos in rp.recv.items():
            ranks[q].send[r] = rp.ghost[pos] - ranks[q].row_lo
    return ShardPlan(world=world, n=n, nparts=nparts, perm=perm, sub_ptr=sub_ptr, coarse_ptr=coarse_ptr,
                     ranks=ranks)


# ---------------------------------------------------------------------------
# per-rank operations and communication
# ---------------------------------------------------------------------------

class RankOps(Protocol):
    """Arithmetic of one rank on its owned block: vectors of n_owned rows
    (internal order), or blocks of n_owned rows by R right-hand sides;
    coarse vectors in paper order, with the same columns."""

    def spmv(self, p_owned, p_ghost): ...                 # q = (A p) on the owned rows
    def local_restrict(self, r_owned): ...                # (z_f, r_c of the owned subdomains)
    def coarse_solve(self, rc_full): ...                  # e_c = A_0^{-1} r_c (replicated)
    def prolong(self, zf_owned, ec_full): ...             # z = z_f + R_0^T e_c on the owned rows
    def sddmm(self, lam_owned, u_owned, u_ghost): ...     # -sum_k lam_k[row_e] u_k[col_e] per owned entry
    def dot(self, a, b): ...                              # a.b: a float, or one per column
    def axpy(self, alpha, x, y): ...                      # y + alpha x (alpha: float, or one per column)
    def copy(self, x): ...
    def zeros_like(self, x): ...
    def gather(self, x, idx): ...                         # x[idx]


class RankFailure(RuntimeError):
    """An exchange of the sharded iteration did not complete: a peer rank
    left or died, or did not join within the process group's timeout.  The
    solve on this rank stops at that exchange (its iterate is not returned);
    the caller decides whether to rebuild the group and start again."""

    def __init__(self, exchange: str, rank: int, cause: BaseException):
        super().__init__(f"{exchange} on rank {rank} did not complete: {cause}")
        self.exchange, self.rank = exchange, rank


class TorchComm:
    """Collectives of the sharded iteration over the default process group
    (gloo on CPU ranks, NCCL on GPUs): vectors travel as float64 tensors.
    ``group`` selects another process group spanning every rank (its
    timeout then bounds each exchange).  A collective that fails (the
    backend reports a closed connection or the group's timeout) is raised
    as RankFailure naming the exchange."""

    def __init__(self, plan: RankPlan, world: int, group=None):
        import torch
        import torch.distributed as dist
        self.torch, self.dist = torch, dist
        self.plan, self.world, self.group = plan, world, group

    def _t(self, x):
        return self.torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64))

    def _run(self, exchange: str, fn):
        """Run the transfers of one exchange (fn holds nothing else: the
        backends report a lost peer and a timeout as plain RuntimeError)."""
        try:
            return fn()
        except RuntimeError as e:
            raise RankFailure(exchange, self.plan.rank, e) from e

    def allreduce(self, values) -> np.ndarray:
        t = self._t(values)
        self._run("all-reduce", lambda: self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group))
        return t.numpy()

    def halo(self, p_owned) -> np.ndarray:
        """Ghost entries of p from their owners (point-to-point)."""
        pl = self.plan
        cols = np.shape(p_owned)[1:]
        out = np.zeros((len(pl.ghost),) + cols)
        sends = {q: self._t(np.asarray(p_owned)[rows]) for q, rows in pl.send.items()}
        bufs = {q: self.torch.empty((len(pos),) + cols, dtype=self.torch.float64) for q, pos in pl.recv.items()}

        def exchange():   # only the transfers: what fails here is the exchange
            reqs = [self.dist.isend(s, dst=q, group=self.group) for q, s in sends.items()]
            reqs += [self.dist.irecv(b, src=q, group=self.group) for q, b in bufs.items()]
            for rq in reqs:
                rq.wait()

        self._run("halo exchange", exchange)
        for q, pos in pl.recv.items():
            out[pos] = bufs[q].numpy()
        return out

    def allgather_coarse(self, rc_owned, coarse_lo: List[int]) -> np.ndarray:
        """The full coarse vector (or block, one column per right-hand side)
        from every rank's contiguous block of rows."""
        sizes = [coarse_lo[r + 1] - coarse_lo[r] for r in range(self.world)]
        width = max(max(sizes), 1)
        rc = np.asarray(rc_owned, dtype=np.float64)
        mine = np.zeros((width,) + rc.shape[1:])
        mine[:len(rc)] = rc
        parts = [self.torch.empty(mine.shape, dtype=self.torch.float64) for _ in range(self.world)]
        self._run("all-gather of r_c", lambda: self.dist.all_gather(parts, self._t(mine), group=self.group))
        return np.concatenate([parts[r].numpy()[:sizes[r]] for r in range(self.world)])


# ---------------------------------------------------------------------------
# the sharded iteration
# ---------------------------------------------------------------------------

@dataclass
class ShardedResult:
    x: object                    # owned rows of the solution (internal order)
    iters: object                # int, or one per column
    relres: object               # recurrence residual / ||f||: float, or one per column
    alphas: list                 # step lengths (one list per column with several)
    betas: list
    collectives: dict


def sharded_pcg(plan: ShardPlan, rank: int, ops: RankOps, comm, f_owned, rtol: float = 1e-8,
                maxit: int = 10000, flexible: bool = False) -> ShardedResult:
    """Preconditioned CG (flexible CG with ``flexible``) from x_0 = 0 on one
    rank's block, with the exchanges of the module docstring; the recurrences
    and the stopping rule (first k with ||r_k|| <= rtol ||f||, recurrence
    residual) are those of the single-rank solve, and the step length and
    beta use the globally reduced dots.

    ``f_owned`` holds the rank's rows of one right-hand side, or of R of
    them as columns.  Each column is its own CG (its own step lengths and
    stop; a converged column keeps its x and r, with step length 0), and
    every exchange carries all columns at once, so an iteration still has
    one halo exchange, two all-reduces and one all-gather.  The scalars
    (one per column) are formed here from the reduced dots."""
    rp = plan.ranks[rank]
    clo = [plan.ranks[r].coarse_lo for r in range(plan.world)] + [plan.ranks[-1].coarse_hi]
    coll = {"halo": 0, "allreduce": 0, "allgather": 0}
    one = np.ndim(f_owned) == 1
    R = 1 if one else int(np.shape(f_owned)[1])
    coef = (lambda v: float(v[0])) if one else (lambda v: v)

    def precond(r):
        zf, rc = ops.local_restrict(r)
        coll["allgather"] += 1
        rc_full = comm.allgather_coarse(rc, clo)
        return ops.prolong(zf, ops.coarse_solve(rc_full))

    def reduce(*dots):
        coll["allreduce"] += 1
        v = comm.allreduce(np.concatenate([np.atleast_1d(np.asarray(d, dtype=np.float64)) for d in dots]))
        return [np.asarray(v[i * R:(i + 1) * R], dtype=np.float64) for i in range(len(dots))]

    def result(x, iters, rr, fn2, alphas, betas):
        rel = np.sqrt(np.divide(rr, fn2, out=np.zeros(R), where=fn2 > 0))
        if one:
            return ShardedResult(x, int(iters[0]), float(rel[0]), alphas[0], betas[0], coll)
        return ShardedResult(x, iters, rel, alphas, betas, coll)

    r = ops.copy(f_owned)
    x = ops.zeros_like(r)
    (fn2,) = reduce(ops.dot(r, r))
    alphas, betas = [[] for _ in range(R)], [[] for _ in range(R)]
    iters = np.zeros(R, dtype=np.int64)
    active = fn2 > 0.0
    rr = fn2.copy()
    if not active.any():
        return result(x, iters, rr, fn2, alphas, betas)
    z = precond(r)
    (rho,) = reduce(ops.dot(r, z))
    p = ops.copy(z)
    k = 0
    while k < maxit and active.any():
        coll["halo"] += 1
        q = ops.spmv(p, comm.halo(p))
        (pq,) = reduce(ops.dot(p, q))
        bad = active & ~(pq > 0.0)
        if bad.any():
            raise FloatingPointError(f"CG breakdown: p^T A p <= 0 (column {int(np.flatnonzero(bad)[0])})")
        alpha = np.divide(rho, pq, out=np.zeros(R), where=active)
        for c in np.flatnonzero(active):
            alphas[c].append(float(alpha[c]))
        x = ops.axpy(coef(alpha), p, x)
        r = ops.axpy(coef(-alpha), q, r)
        k += 1
        z = precond(r)
        rr_k, rz, zq = reduce(ops.dot(r, r), ops.dot(r, z), ops.dot(z, q))
        rr = np.where(active, rr_k, rr)
        done = active & (rr_k <= rtol * rtol * fn2)
        iters[done] = k
        active = active & ~done
        # flexible: z_{k+1}^T (r_{k+1} - r_k) = -alpha z_{k+1}^T q_k
        beta = np.divide(-alpha * zq if flexible else rz, rho, out=np.zeros(R), where=active)
        for c in np.flatnonzero(active):
            betas[c].append(float(beta[c]))
        rho = np.where(active, rz, rho)
        p = ops.axpy(coef(beta), p, z)
    iters[active] = k
    return result(x, iters, rr, fn2, alphas, betas)


def sharded_adjoint(plan: ShardPlan, rank: int, ops: RankOps, comm, g_owned, u_owned, rtol: float = 1e-8,
                    maxit: int = 10000):
    """Adjoint of u = A^{-1} f for a loss L(u) with dL/du = g, on one rank's
    block: lambda = A^{-1} g by the sharded PCG (A is symmetric, so the same
    preconditioner serves), one more halo exchange (the ghost entries of u),
    then dL/dA on the rank's own rows, dvals[e] = -sum_k lambda_k[row_e]
    u_k[col_e], in the rank's entry order (``plan.ranks[rank].entry`` maps
    each to the caller's CSR entry); dL/df = lambda.  Returns (lambda owned
    rows, dvals, the PCG result)."""
    res = sharded_pcg(plan, rank, ops, comm, g_owned, rtol=rtol, maxit=maxit)
    res.collectives["halo"] += 1
    u_ghost = comm.halo(u_owned)
    return res.x, ops.sddmm(res.x, u_owned, u_ghost), res
