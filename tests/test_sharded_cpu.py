"""The sharded solve phase on CPU ranks (gloo): contiguous subdomain ranges
per rank, a halo exchange of p before each SpMV, all-reduces of the dots,
an all-gather of r_c before the replicated coarse solve.  Its iterates
equal the single-rank solve's (the oracle's PCG and flexible CG) to 1e-12
at world sizes 2 and 4; the plan's ghost, send and receive lists are
checked by brute force.  A lost peer (one that exits, never joins an
exchange, or leaves between iterations) ends the other ranks' solve with
RankFailure at the exchange that could not complete.  The sharded adjoint
(lambda on every rank, dL/dA on its entries) equals the oracle's."""

import os
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

from workloads import make_small_2d, make_small_3d

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = {
    "2d": lambda: make_small_2d(side=40, bs=8, m=3, std=2.0, sigma=3.0, seed=61, ny=33),
    "3d": lambda: make_small_3d(side=12, bs=4, m=4, std=2.0, sigma=2.0, seed=62),
}


def _plan(w, world):
    from oracle import OracleAMS, csr_to_scipy
    from paper_2606_04864_gb300.sharded import make_plan
    o = OracleAMS(csr_to_scipy(w.rowptr, w.colind, w.vals), w.part, w.nparts, w.m)
    return o, make_plan(w.rowptr, w.colind, w.vals, w.part, w.nparts, o.m_i, world)


@pytest.mark.parametrize("world", [1, 2, 3, 4, 7])
@pytest.mark.parametrize("case", list(CASES))
def test_plan_ranges_ghosts_and_exchange_lists(case, world):
    w = CASES[case]()
    o, plan = _plan(w, world)
    n = w.n
    assert (plan.perm == o.perm).all() and (plan.sub_ptr == o.sub_ptr).all()
    iperm = np.empty(n, dtype=np.int64)
    iperm[plan.perm] = np.arange(n)
    sizes = [rp.n_owned for rp in plan.ranks]
    assert sum(sizes) == n and plan.ranks[0].row_lo == 0 and plan.ranks[-1].row_hi == n
    assert max(sizes) - min(sizes) <= 2 * max(np.diff(plan.sub_ptr))      # balanced to a subdomain
    A = __import__("scipy.sparse", fromlist=["csr_matrix"]).csr_matrix((w.vals, w.colind, w.rowptr), shape=(n, n))
    P = A[plan.perm][:, plan.perm].tocsr()                                  # internal order
    for rp in plan.ranks:
        blk = P[rp.row_lo:rp.row_hi]
        cols = np.unique(blk.indices)
        ghost = cols[(cols < rp.row_lo) | (cols >= rp.row_hi)]
        assert np.array_equal(ghost, rp.ghost)
        # the rank's rows of A in owned-then-ghost numbering reproduce the block
        full = np.concatenate([np.arange(rp.row_lo, rp.row_hi), rp.ghost])
        L = __import__("scipy.sparse", fromlist=["csr_matrix"]).csr_matrix(
            (rp.vals, rp.colind, rp.rowptr), shape=(rp.n_owned, len(full)))
        x = np.random.default_rng(rp.rank).standard_normal(n)
        assert np.allclose(L @ x[full], blk @ x, rtol=0, atol=1e-14 * np.abs(blk @ x).max())
        # receives are exactly the ghosts, each from its owner; sends mirror them
        got = np.concatenate([rp.ghost[pos] for pos in rp.recv.values()]) if rp.recv else np.zeros(0, int)
        assert np.array_equal(np.sort(got), rp.ghost)
        for q, pos in rp.recv.items():
            src = plan.ranks[q]
            assert ((rp.ghost[pos] >= src.row_lo) & (rp.ghost[pos] < src.row_hi)).all()
            assert np.array_equal(src.send[rp.rank] + src.row_lo, rp.ghost[pos])
    # every caller CSR entry sits on exactly one rank, with its value
    ent = np.concatenate([rp.entry for rp in plan.ranks])
    assert np.array_equal(np.sort(ent), np.arange(w.nnz))
    for rp in plan.ranks:
        assert np.array_equal(rp.vals, w.vals[rp.entry])
    # coarse blocks are contiguous and cover N_c in rank order
    assert plan.ranks[0].coarse_lo == 0 and plan.ranks[-1].coarse_hi == o.Nc
    for a, b in zip(plan.ranks[:-1], plan.ranks[1:]):
        assert a.coarse_hi == b.coarse_lo and a.sub_hi == b.sub_lo


def _worker(rank, world, port, case, flexible, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2606_04864_gb300.sharded import TorchComm, sharded_pcg
        from tests.sharded_oracle_ops import OracleRankOps
        w = CASES[case]()
        o, plan = _plan(w, world)
        rp = plan.ranks[rank]
        f_owned = w.rhs[0][plan.perm[rp.row_lo:rp.row_hi]]
        res = sharded_pcg(plan, rank, OracleRankOps(o, plan, rank), TorchComm(rp, world), f_owned,
                          rtol=1e-10, flexible=flexible)
        out[rank] = (np.asarray(res.x), res.iters, res.alphas, res.betas, res.collectives)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("flexible", [False, True])
@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("case", list(CASES))
def test_sharded_iterates_equal_single_rank(case, world, flexible):
    from oracle import OracleAMS, csr_to_scipy, pcg
    w = CASES[case]()
    A = csr_to_scipy(w.rowptr, w.colind, w.vals)
    o = OracleAMS(A, w.part, w.nparts, w.m)
    ref = pcg(A, w.rhs[0], o.apply, rtol=1e-10, flexible=flexible)
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 20000 + (os.getpid() * 7 + world * 131 + (5 if flexible else 0) + len(case)) % 20000
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, flexible, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    x = np.concatenate([out[r][0] for r in range(world)])
    u = np.empty(w.n)
    u[o.perm] = x
    assert all(out[r][1] == ref.iters for r in range(world))
    assert np.linalg.norm(u - ref.u) <= 1e-12 * np.linalg.norm(ref.u)
    for r in range(world):
        assert np.allclose(out[r][2], ref.alphas, rtol=1e-12, atol=0)
        assert np.allclose(out[r][3], ref.betas, rtol=1e-10, atol=1e-14)
        c = out[r][4]
        # per iteration: one halo exchange, two all-reduces, one all-gather
        assert c["halo"] == ref.iters and c["allreduce"] == 2 + 2 * ref.iters
        assert c["allgather"] == 1 + ref.iters


def _block_rhs(w):
    """Four right-hand sides as columns: the workload's, a zero column, a
    seeded N(0,1) one and the first scaled by 1e-3 (its own stop, the same
    step lengths)."""
    g = np.random.default_rng(5).standard_normal(w.n)
    return np.column_stack([w.rhs[0], np.zeros(w.n), g, 1e-3 * w.rhs[0]])


def _block_worker(rank, world, port, case, flexible, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2606_04864_gb300.sharded import TorchComm, sharded_pcg
        from tests.sharded_oracle_ops import OracleRankOps
        w = CASES[case]()
        o, plan = _plan(w, world)
        rp = plan.ranks[rank]
        F = _block_rhs(w)[plan.perm[rp.row_lo:rp.row_hi]]
        res = sharded_pcg(plan, rank, OracleRankOps(o, plan, rank), TorchComm(rp, world), F,
                          rtol=1e-10, flexible=flexible)
        out[rank] = (np.asarray(res.x), list(res.iters), res.alphas, res.betas, res.collectives)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("flexible", [False, True])
@pytest.mark.parametrize("world", [2, 3])
def test_sharded_block_of_rhs_equals_single_rank_per_column(world, flexible):
    """Several right-hand sides on shared exchanges: every column takes the
    single-rank oracle solve's iteration count, step lengths and solution
    (the zero column none), and an iteration still has one halo exchange,
    two all-reduces and one all-gather, however many columns are active."""
    from oracle import OracleAMS, csr_to_scipy, pcg
    case = "3d"
    w = CASES[case]()
    A = csr_to_scipy(w.rowptr, w.colind, w.vals)
    o = OracleAMS(A, w.part, w.nparts, w.m)
    F = _block_rhs(w)
    refs = [pcg(A, F[:, c], o.apply, rtol=1e-10, flexible=flexible) for c in range(F.shape[1])]
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 20000 + (os.getpid() * 13 + world * 151 + (7 if flexible else 0)) % 20000
    procs = [ctx.Process(target=_block_worker, args=(r, world, port, case, flexible, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    X = np.concatenate([out[r][0] for r in range(world)])
    U = np.empty_like(X)
    U[o.perm] = X
    its = max(ref.iters for ref in refs)
    assert refs[1].iters == 0 and refs[0].iters == refs[3].iters
    for r in range(world):
        assert out[r][1] == [ref.iters for ref in refs]
        c = out[r][4]
        assert c["halo"] == its and c["allreduce"] == 2 + 2 * its and c["allgather"] == 1 + its
        for col, ref in enumerate(refs):
            assert np.allclose(out[r][2][col], ref.alphas, rtol=1e-12, atol=0)
            assert np.allclose(out[r][3][col], ref.betas, rtol=1e-10, atol=1e-14)
    for col, ref in enumerate(refs):
        assert np.linalg.norm(U[:, col] - ref.u) <= 1e-12 * max(np.linalg.norm(ref.u), 1e-300)
    assert not U[:, 1].any()


def _adjoint_inputs(w, A, o, ncols):
    """The forward solutions u (oracle CG to 1e-12) of the workload's
    right-hand side and of a seeded N(0,1) one, and seeded loss gradients g,
    as columns."""
    from oracle import pcg
    rng = np.random.default_rng(9)
    F = np.column_stack([w.rhs[0], rng.standard_normal(w.n)])[:, :ncols]
    U = np.column_stack([pcg(A, F[:, k], o.apply, rtol=1e-12).u for k in range(ncols)])
    G = rng.standard_normal((w.n, ncols))
    return U, G


def _adjoint_worker(rank, world, port, ncols, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import csr_to_scipy
        from paper_2606_04864_gb300.sharded import TorchComm, sharded_adjoint
        from tests.sharded_oracle_ops import OracleRankOps
        w = CASES["2d"]()
        o, plan = _plan(w, world)
        U, G = _adjoint_inputs(w, csr_to_scipy(w.rowptr, w.colind, w.vals), o, ncols)
        rp = plan.ranks[rank]
        rows = plan.perm[rp.row_lo:rp.row_hi]
        g, u = (G[rows, 0], U[rows, 0]) if ncols == 1 else (G[rows], U[rows])
        lam, dvals, res = sharded_adjoint(plan, rank, OracleRankOps(o, plan, rank), TorchComm(rp, world), g, u,
                                          rtol=1e-10)
        out[rank] = (np.asarray(lam), np.asarray(dvals), res.iters, res.collectives)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ncols", [1, 2])
@pytest.mark.parametrize("world", [2, 3])
def test_sharded_adjoint_matches_oracle_gradient(world, ncols):
    """The sharded adjoint: lambda on every rank's rows and dL/dA on its
    entries, mapped back to the caller's CSR entries by the plan, equal the
    oracle's adjoint (summed over the columns) to 1e-10; one halo exchange
    more than the solve."""
    from oracle import OracleAMS, adjoint_gradient, csr_to_scipy
    w = CASES["2d"]()
    A = csr_to_scipy(w.rowptr, w.colind, w.vals)
    o = OracleAMS(A, w.part, w.nparts, w.m)
    U, G = _adjoint_inputs(w, A, o, ncols)
    refs = [adjoint_gradient(A, U[:, k], G[:, k], o.apply, rtol=1e-10) for k in range(ncols)]
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 20000 + (os.getpid() * 17 + world * 173 + ncols * 29) % 20000
    procs = [ctx.Process(target=_adjoint_worker, args=(r, world, port, ncols, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    _, plan = _plan(w, world)
    dv = np.full(w.nnz, np.nan)
    for r in range(world):
        rp = plan.ranks[r]
        lam, dvals, iters, coll = out[r]
        rows = plan.perm[rp.row_lo:rp.row_hi]
        for k, ref in enumerate(refs):
            lk = lam if ncols == 1 else lam[:, k]
            assert np.linalg.norm(lk - ref[0][rows]) <= 1e-10 * np.linalg.norm(ref[0][rows])
            assert (iters if ncols == 1 else iters[k]) == ref[2].iters
        its = max(ref[2].iters for ref in refs)
        assert coll["halo"] == its + 1
        dv[rp.entry] = dvals
    expect = sum(ref[1] for ref in refs)
    assert not np.isnan(dv).any()          # every caller entry belongs to exactly one rank
    assert np.linalg.norm(dv - expect) <= 1e-10 * np.linalg.norm(expect)


def _failure_worker(rank, world, port, mode, out):
    """Rank 1 leaves the solve in one of three ways; rank 0 solves and
    reports how its solve ended.  Every exchange runs in a group with a
    3 s timeout (the default group keeps a long one for the rendezvous)."""
    import datetime
    import time
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=120))
    group = dist.new_group(list(range(world)), timeout=datetime.timedelta(seconds=3))
    from paper_2606_04864_gb300.sharded import RankFailure, TorchComm, sharded_pcg
    from tests.sharded_oracle_ops import OracleRankOps
    w = CASES["2d"]()
    o, plan = _plan(w, world)
    rp = plan.ranks[rank]
    f_owned = w.rhs[0][plan.perm[rp.row_lo:rp.row_hi]]
    comm = TorchComm(rp, world, group=group)
    if rank == 1:
        if mode == "exits":              # gone before the solve's first exchange
            os._exit(0)
        if mode == "never_joins":        # alive, but joins no exchange
            time.sleep(40)
            os._exit(0)
        # "leaves_after_3": three full iterations, then gone between steps
        sharded_pcg(plan, rank, OracleRankOps(o, plan, rank), comm, f_owned, rtol=1e-10, maxit=3)
        os._exit(0)
    t0 = time.monotonic()
    try:
        sharded_pcg(plan, rank, OracleRankOps(o, plan, rank), comm, f_owned, rtol=1e-10)
        out[rank] = ("finished", time.monotonic() - t0, "")
    except RankFailure as e:
        out[rank] = ("RankFailure", time.monotonic() - t0, e.exchange)
    os._exit(0)   # the group is broken: leave without a teardown that talks to the lost peer


@pytest.mark.parametrize("mode, exchange", [("exits", "all-reduce"), ("never_joins", "all-reduce"),
                                            ("leaves_after_3", "halo exchange")])
def test_lost_rank_ends_the_solve_with_rank_failure(mode, exchange):
    """Failure detection on the host: a peer that exits, one that never
    joins, and one that leaves after three iterations each end the other
    rank's solve with RankFailure at the exchange that could not complete,
    within the group's timeout instead of hanging."""
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 20000 + (os.getpid() * 11 + 17 * len(mode)) % 20000
    procs = [ctx.Process(target=_failure_worker, args=(r, 2, port, mode, out)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        procs[0].join(120)
        assert procs[0].exitcode == 0, "the surviving rank did not finish"
    finally:
        for p in procs:
            p.join(0 if p is procs[1] and mode == "never_joins" else 60)
            if p.is_alive():
                p.kill()
                p.join()
    status, seconds, where = out[0]
    assert status == "RankFailure", (status, seconds)
    assert where == exchange
    if mode == "never_joins":
        assert 2.5 <= seconds < 30.0   # the group's 3 s timeout, not the idle peer's 40 s sleep
    else:
        assert seconds < 10.0          # a closed connection is reported at once
