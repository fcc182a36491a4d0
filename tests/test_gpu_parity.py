"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Sizes are small enough for the oracle to finish in seconds while still
spanning several 32-row tiles, ragged last tiles, uneven subdomains and
multi-level coarse trees.  Tolerances: index maps bit-exact; FP64 path
relative solution error <= 1e-10 and iterations within 2 of the oracle;
reduced-precision paths <= 1e-6 against the FP64 oracle.
"""

import numpy as np
import pytest
import scipy.linalg as la

from oracle import OracleAMS, csr_to_scipy, pcg
from workloads import make_grf2d_64, make_small_2d, make_small_3d

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2606_04864_gb300 import AmsBatchedSolver, AmsError, AmsSolver  # noqa: E402


def _A(w):
    return csr_to_scipy(w.rowptr, w.colind, w.vals)


def _solver(w, **kw):
    return AmsSolver(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m, **kw)


def _proj(Psi, s):
    return Psi @ Psi.T @ np.diag(s)


CASES = {
    "grf2d_64": lambda: make_grf2d_64(),
    "2d_ragged": lambda: make_small_2d(side=45, bs=10, m=3, std=2.0, sigma=3.0, seed=31, ny=37),
    "3d_b8": lambda: make_small_3d(side=16, bs=8, m=6, std=2.5, sigma=3.0, seed=32),
    "3d_ragged": lambda: make_small_3d(side=13, bs=5, m=4, std=2.0, sigma=2.0, seed=33),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    w = CASES[request.param]()
    A = _A(w)
    o = OracleAMS(A, w.part, w.nparts, w.m)
    return request.param, w, A, o


def test_index_maps_bit_exact(case):
    name, w, A, o = case
    s = _solver(w, precision="fp64")
    perm, sub_ptr = s.index_maps()
    assert (perm == o.perm).all()
    assert (sub_ptr == o.sub_ptr).all()


def test_eigenpairs_match_oracle(case):
    name, w, A, o = case
    s = _solver(w, precision="fp64")
    mi, lams, psis = s.coarse_basis()
    assert list(mi) == list(o.m_i)
    info = s.info()
    assert info["eig_max_residual"] <= 1e-11
    for i, dofs in enumerate(o.sub_dofs):
        lam_o = o.lams[i][:mi[i]]
        assert np.abs(lams[i] - lam_o).max() <= 1e-11 * max(1.0, np.abs(lam_o).max())
        _, _, sw = __import__("oracle").local_matrices(A, dofs)
        G = psis[i].T @ (sw[:, None] * psis[i])
        assert np.abs(G - np.eye(mi[i])).max() <= 1e-11
        P1, P2 = _proj(psis[i], sw), _proj(o.Psis[i], sw)
        assert np.abs(P1 - P2).max() <= 1e-8 * max(1.0, np.abs(P2).max())


def test_coarse_matrix_matches_oracle(case):
    name, w, A, o = case
    s = _solver(w, precision="fp64")
    A0 = s.coarse_matrix()
    # basis signs may differ: compare the sign-invariant quantity |A0_ij|
    # plus the spectrum (A0 is D A0_oracle D for a diagonal sign matrix D)
    ev_g = np.linalg.eigvalsh(A0)
    ev_o = np.linalg.eigvalsh(o.A0)
    assert np.abs(ev_g - ev_o).max() <= 1e-10 * ev_o.max()
    assert np.abs(np.abs(A0) - np.abs(o.A0)).max() <= 1e-9 * np.abs(o.A0).max()


FACTOR_CASES = {
    # several 64-row tiles, deep nested-dissection trees, tiles straddling
    # tree nodes, a ragged last tile
    "2d_2400": lambda: make_small_2d(side=160, bs=8, m=6, std=2.0, sigma=3.0, seed=41),
    "3d_4000": lambda: make_small_3d(side=40, bs=4, m=4, std=2.0, sigma=2.0, seed=42),
    "2d_ragged_b10_m11": lambda: make_small_2d(side=111, bs=10, m=11, std=2.0, sigma=3.0, seed=43, ny=111),
}


@pytest.mark.parametrize("name", list(FACTOR_CASES))
def test_coarse_factor_inverse_matches_dense_cholesky(name):
    """The tile Cholesky factor of A_0 and its inverse, computed only on the
    tiles that the nested-dissection order keeps, against LAPACK's dense
    Cholesky of the same A_0 and a dense triangular inverse."""
    w = FACTOR_CASES[name]()
    s = _solver(w, precision="fp64")
    A0 = s.coarse_matrix()
    X, order = s.coarse_factor_inverse()
    nc = len(order)
    assert nc == A0.shape[0] and nc > 1000
    assert (np.sort(order) == np.arange(nc)).all()
    A0nd = A0[np.ix_(order, order)]
    L = np.linalg.cholesky(A0nd)
    Xref = la.solve_triangular(L, np.eye(nc), lower=True)
    assert not np.triu(X, 1).any()
    err = np.abs(X - Xref).max() / np.abs(Xref).max()
    ident = np.abs(X @ A0nd @ X.T - np.eye(nc)).max()
    print(f"{name}: N_c={nc} max|X-Xref|/max|Xref|={err:.2e} max|X A0 X^T - I|={ident:.2e}")
    assert err <= 1e-11
    assert ident <= 1e-11
    info = s.info()
    assert 0.0 < info["coarse_factor_gflop"] < 2 * nc ** 3 / 3 * 1e-9


def test_spmv_matches_scipy(case):
    name, w, A, o = case
    s = _solver(w, precision="fp64")
    x = np.random.default_rng(1).standard_normal((3, w.n))
    y = s.spmv(x)
    ref = (A @ x.T).T
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 2e-5), ("fp32_bf16", 2e-5)])
def test_preconditioner_apply_matches_oracle(case, prec, tol):
    name, w, A, o = case
    rnd = {"fp64": None, "fp32": "fp32", "fp32_bf16": "bf16"}[prec]
    orc = o if rnd is None else OracleAMS(A, w.part, w.nparts, w.m, basis_round=rnd)
    s = _solver(w, precision=prec)
    r = np.random.default_rng(2).standard_normal((2, w.n))
    z = s.apply_preconditioner(r)
    for k in range(2):
        zr = orc.apply(r[k])
        assert np.linalg.norm(z[k] - zr) <= tol * np.linalg.norm(zr), (prec, np.linalg.norm(z[k] - zr) / np.linalg.norm(zr))


def test_fp64_pcg_matches_oracle(case):
    name, w, A, o = case
    ref = pcg(A, w.rhs[0], o.apply, rtol=1e-8)
    s = _solver(w, precision="fp64")
    u, its, rel = s.solve(w.rhs[0], rtol=1e-8)
    assert abs(int(its[0]) - ref.iters) <= 2
    assert np.linalg.norm(u - ref.u) <= 1e-10 * np.linalg.norm(ref.u)
    assert np.linalg.norm(w.rhs[0] - A @ u) <= 1.5e-8 * np.linalg.norm(w.rhs[0])


@pytest.mark.parametrize("prec", ["fp32", "fp32_bf16"])
def test_mixed_fcg_matches_fp64_oracle(case, prec):
    name, w, A, o = case
    ref = pcg(A, w.rhs[0], o.apply, rtol=1e-8)
    tight = pcg(A, w.rhs[0], o.apply, rtol=1e-13)
    s = _solver(w, precision=prec)
    u, its, rel = s.solve(w.rhs[0], rtol=1e-8)
    assert abs(int(its[0]) - ref.iters) <= 2, (its, ref.iters)
    floor = np.linalg.norm(ref.u - tight.u) / np.linalg.norm(tight.u)
    err = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    assert err <= max(1e-6, 10 * floor), (err, floor)
    assert np.linalg.norm(w.rhs[0] - A @ u) <= 1.5e-8 * np.linalg.norm(w.rhs[0])


def test_multi_rhs_each_column_matches_oracle():
    w = make_small_3d(side=12, bs=4, m=4, std=2.0, sigma=2.0, seed=40, nrhs=5, rhs_kind="normal")
    A = _A(w)
    o = OracleAMS(A, w.part, w.nparts, w.m)
    for prec, tol in [("fp64", 1e-10), ("fp32_bf16", 1e-6)]:
        s = _solver(w, precision=prec)
        u, its, rel = s.solve(w.rhs, rtol=1e-8)
        for k in range(w.nrhs):
            ref = pcg(A, w.rhs[k], o.apply, rtol=1e-8)
            assert abs(int(its[k]) - ref.iters) <= 2
            assert np.linalg.norm(u[k] - ref.u) <= tol * np.linalg.norm(ref.u)


def test_thirty_two_rhs_device_pointers():
    w = make_small_2d(side=40, bs=8, m=4, std=2.0, seed=41, nrhs=32, rhs_kind="normal")
    A = _A(w)
    s = _solver(w, precision="fp32_bf16", device=True)
    f = torch.as_tensor(w.rhs, device="cuda")
    u, its, rel = s.solve(f, rtol=1e-8)
    u = u.cpu().numpy()
    R = w.rhs - (A @ u.T).T
    assert (np.linalg.norm(R, axis=1) <= 1.5e-8 * np.linalg.norm(w.rhs, axis=1)).all()
    assert (rel <= 1e-8).all()


def test_adjoint_matches_oracle():
    w = make_small_2d(side=24, bs=6, m=3, std=2.0, seed=42)
    A = _A(w)
    o = OracleAMS(A, w.part, w.nparts, w.m)
    s = _solver(w, precision="fp64")
    u, _, _ = s.solve(w.rhs[0], rtol=1e-12)
    g = np.random.default_rng(3).standard_normal(w.n)
    lam, dvals, its = s.solve_adjoint(g, u, rtol=1e-12)
    from oracle import adjoint_gradient
    lam_o, dv_o, _ = adjoint_gradient(A, u, g, o.apply, rtol=1e-12)
    assert np.linalg.norm(lam - lam_o) <= 1e-9 * np.linalg.norm(lam_o)
    assert np.abs(dvals - dv_o).max() <= 1e-9 * np.abs(dv_o).max()


def test_batched_uneven_systems_match_oracle():
    ws = [make_small_2d(side=20, bs=8, m=4, std=2.0, seed=50),
          make_small_3d(side=9, bs=4, m=3, std=2.5, seed=51),
          make_small_2d(side=33, bs=8, m=5, std=2.0, seed=52, ny=17)]
    systems = [(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m) for w in ws]
    nrhs = 3
    rhs = [np.random.default_rng(60 + i).standard_normal((nrhs, w.n)) for i, w in enumerate(ws)]
    for prec, tol in [("fp64", 1e-10), ("fp32_bf16", 1e-6)]:
        b = AmsBatchedSolver(systems, precision=prec)
        u, its, rel = b.solve(b.pack(rhs), nrhs, rtol=1e-8)
        us = b.unpack(u, nrhs)
        for i, w in enumerate(ws):
            A = _A(w)
            o = OracleAMS(A, w.part, w.nparts, w.m)
            for k in range(nrhs):
                ref = pcg(A, rhs[i][k], o.apply, rtol=1e-8)
                assert abs(int(its[i, k]) - ref.iters) <= 2
                assert np.linalg.norm(us[i][k] - ref.u) <= tol * np.linalg.norm(ref.u)


@pytest.mark.parametrize("nrhs", [8, 16])
def test_batched_mixed_band_widths_many_rhs(nrhs):
    """Systems whose subdomains have different band widths (8x8 2-D blocks:
    one 32-row band tile; 8^3 3-D blocks: two) with 8 and 16 right-hand
    sides, where the tensor-core local solve launches once per band-width
    group over an index list: iterations and solutions against the oracle."""
    ws = [make_small_2d(side=40, bs=8, m=4, std=2.0, seed=53),
          make_small_3d(side=16, bs=8, m=6, std=2.5, seed=54),
          make_small_2d(side=24, bs=8, m=5, std=2.0, seed=55, ny=41)]
    systems = [(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m) for w in ws]
    rhs = [np.random.default_rng(70 + i).standard_normal((nrhs, w.n)) for i, w in enumerate(ws)]
    refs = []
    for i, w in enumerate(ws):
        A = _A(w)
        o = OracleAMS(A, w.part, w.nparts, w.m, basis_round="bf16")
        refs.append([pcg(A, rhs[i][k], o.apply, rtol=1e-8) for k in range(nrhs)])
    b = AmsBatchedSolver(systems, precision="fp32_bf16")
    assert b.info()["max_band_tiles"] == 2
    u, its, rel = b.solve(b.pack(rhs), nrhs, rtol=1e-8)
    buf = np.empty_like(u)
    u2, _, _ = b.solve(b.pack(rhs), nrhs, rtol=1e-8, out=buf)   # into a caller buffer: the same solve
    assert u2 is buf and np.array_equal(buf, u)
    us = b.unpack(u, nrhs)
    for i, w in enumerate(ws):
        for k in range(nrhs):
            assert abs(int(its[i, k]) - refs[i][k].iters) <= 2, (i, k, its[i, k], refs[i][k].iters)
            assert np.linalg.norm(us[i][k] - refs[i][k].u) <= 1e-6 * np.linalg.norm(refs[i][k].u)


@pytest.mark.parametrize("prec", ["fp64", "fp32_bf16"])
def test_fewer_rhs_after_more_replays_no_stale_buffers(prec):
    """A solve with fewer right-hand sides after one with more: the larger
    solve grows the work buffers, and the iteration-loop graph of the smaller
    count, captured before, must not replay on the freed ones.  The same
    solve before and after (with an apply and an SpMV between) is bit-equal,
    and matches the oracle."""
    w = make_small_2d(side=45, bs=10, m=3, std=2.0, sigma=3.0, seed=31, ny=37)
    A = _A(w)
    f = np.random.default_rng(6).standard_normal((32, w.n))
    s = _solver(w, precision=prec)
    u1, i1, _ = s.solve(f[:1], rtol=1e-8)
    u32, i32, _ = s.solve(f, rtol=1e-8)
    s.apply_preconditioner(f[:4])
    s.spmv(f[:2])
    u1b, i1b, _ = s.solve(f[:1], rtol=1e-8)
    assert np.array_equal(np.asarray(u1), np.asarray(u1b)) and int(i1[0]) == int(i1b[0])
    ref = pcg(A, f[0], OracleAMS(A, w.part, w.nparts, w.m).apply, rtol=1e-8)
    tol = 1e-10 if prec == "fp64" else 1e-6
    assert np.linalg.norm(np.atleast_2d(u1b)[0] - ref.u) <= tol * np.linalg.norm(ref.u)
    assert np.linalg.norm(np.asarray(u32)[0] - ref.u) <= tol * np.linalg.norm(ref.u)


# ------------------------------------------------------------- edge cases

def test_isolated_dofs_and_tiny_subdomains():
    """Subdomains of one dof (no in-subdomain neighbour: S_jj = A_jj) and
    m >= n_i (every local mode kept)."""
    w = make_small_2d(side=10, bs=3, m=4, std=1.0, seed=70)
    part = w.part.copy()
    part = np.where(np.arange(w.n) % 17 == 0, w.nparts + np.arange(w.n) // 17, part)
    uniq, part = np.unique(part, return_inverse=True)
    part = part.astype(np.int32)
    A = _A(w)
    o = OracleAMS(A, part, len(uniq), 4)
    ref = pcg(A, w.rhs[0], o.apply, rtol=1e-8)
    s = AmsSolver(w.rowptr, w.colind, w.vals, part, len(uniq), 4, precision="fp64")
    u, its, rel = s.solve(w.rhs[0], rtol=1e-8)
    assert abs(int(its[0]) - ref.iters) <= 2
    assert np.linalg.norm(u - ref.u) <= 1e-10 * np.linalg.norm(ref.u)


def test_block_jacobi_m0_and_single_subdomain():
    w = make_small_2d(side=16, bs=4, m=0, std=2.0, seed=71)
    A = _A(w)
    o = OracleAMS(A, w.part, w.nparts, 0, coarse=False)
    ref = pcg(A, w.rhs[0], o.apply, rtol=1e-8)
    s = _solver(w, precision="fp64")
    u, its, _ = s.solve(w.rhs[0], rtol=1e-8)
    assert abs(int(its[0]) - ref.iters) <= 2
    assert np.linalg.norm(u - ref.u) <= 1e-10 * np.linalg.norm(ref.u)
    # one subdomain: the local solve is exact, so local-only CG takes one
    # iteration; adding the coarse term makes M^{-1}A = I + (A-orthogonal
    # projector onto the coarse space), eigenvalues {1, 2}: two iterations
    w1 = make_small_2d(side=16, bs=16, m=2, std=2.0, seed=72)
    s1 = _solver(w1, precision="fp64", coarse=False)
    u1, its1, _ = s1.solve(w1.rhs[0], rtol=1e-10)
    assert its1[0] == 1
    s2 = _solver(w1, precision="fp64")
    u2, its2, _ = s2.solve(w1.rhs[0], rtol=1e-10)
    assert its2[0] == 2


def test_zero_rhs_and_maxit():
    w = make_small_2d(side=16, bs=4, m=2, std=2.0, seed=73)
    s = _solver(w, precision="fp64")
    u, its, rel = s.solve(np.zeros(w.n), rtol=1e-8)
    assert its[0] == 0 and np.all(u == 0)
    s2 = _solver(w, precision="fp64", maxit=2)
    with pytest.raises(AmsError) as e:
        s2.solve(w.rhs[0], rtol=1e-12)
    assert e.value.status == 4
    u2, its2, _ = s2.solve(w.rhs[0], rtol=1e-12, allow_not_converged=True)
    assert its2[0] == 2 and np.isfinite(u2).all()


def test_invalid_inputs_are_rejected():
    w = make_small_2d(side=8, bs=4, m=2, seed=74)
    bad = w.vals.copy()
    bad[w.rowptr[3] + 0] *= 1.5            # break symmetry
    with pytest.raises(AmsError) as e:
        AmsSolver(w.rowptr, w.colind, bad, w.part, w.nparts, 2)
    assert e.value.status == 1
    p = w.part.copy()
    p[0] = w.nparts + 3
    with pytest.raises(AmsError) as e:
        AmsSolver(w.rowptr, w.colind, w.vals, p, w.nparts, 2)
    assert e.value.status == 1
    with pytest.raises(AmsError) as e:                 # empty subdomain
        AmsSolver(w.rowptr, w.colind, w.vals, w.part, w.nparts + 1, 2)
    assert e.value.status == 1
    neg = w.vals.copy()
    diag = [w.rowptr[i] + list(w.colind[w.rowptr[i]:w.rowptr[i + 1]]).index(i) for i in range(w.n)]
    neg[diag[5]] = -1.0
    with pytest.raises(AmsError) as e:
        AmsSolver(w.rowptr, w.colind, neg, w.part, w.nparts, 2)
    assert e.value.status == 2
    # indefinite but with positive diagonal: caught by a local Cholesky pivot
    ind = w.vals.copy()
    for i in range(w.n):
        for t in range(w.rowptr[i], w.rowptr[i + 1]):
            if w.colind[t] != i:
                ind[t] *= 3.0
    with pytest.raises(AmsError) as e:
        AmsSolver(w.rowptr, w.colind, ind, w.part, w.nparts, 2)
    assert e.value.status == 2


@pytest.mark.parametrize("prec", ["fp64", "fp32_bf16"])
def test_autotuned_launch_shapes_give_the_same_solve(prec):
    """Launch shapes change block ranges and ring depths, not the arithmetic
    of any row: an autotuned handle and one on the default shapes agree."""
    w = make_small_2d(side=96, bs=16, m=4, std=2.0, sigma=3.0, seed=43, nrhs=3, rhs_kind="normal")
    a = _solver(w, precision=prec, autotune=True)
    b = _solver(w, precision=prec, autotune=False)
    ua, ia, _ = a.solve(w.rhs, rtol=1e-8)
    ub, ib, _ = b.solve(w.rhs, rtol=1e-8)
    assert (np.abs(ia.astype(int) - ib.astype(int)) <= 2).all()
    tol = 1e-10 if prec == "fp64" else 1e-6
    assert np.linalg.norm(ua - ub) <= tol * np.linalg.norm(ub)
    # a second solve reuses the tuned shapes
    ua2, ia2, _ = a.solve(w.rhs, rtol=1e-8)
    assert (ia2 == ia).all() and np.array_equal(ua2, ua)


def test_set_launch_shape_is_validated_and_kept():
    """A fixed launch shape is reported back, survives the first solve (the
    autotuner leaves it), replaces the captured iteration graph, and gives
    the solve of the default shapes; invalid shapes are refused."""
    from paper_2606_04864_gb300._lib import AmsError
    w = make_small_2d(side=96, bs=16, m=4, std=2.0, sigma=3.0, seed=45, nrhs=3, rhs_kind="normal")
    a = _solver(w, precision="fp32_bf16", autotune=True)
    assert not a.launch_shape(3)["fixed"]
    a.set_launch_shape(3, bps_elem=3, bps_sub=6, depth=2, nr=2)
    assert a.launch_shape(4) == {"bps_elem": 3, "bps_sub": 6, "depth": 2, "nr": 2, "l2mode": 0, "l2keep": 0,
                                 "fixed": True}
    ua, ia, _ = a.solve(w.rhs, rtol=1e-8)
    assert a.launch_shape(3) == {"bps_elem": 3, "bps_sub": 6, "depth": 2, "nr": 2, "l2mode": 0, "l2keep": 0,
                                 "fixed": True}
    a.set_launch_shape(3, bps_elem=6, depth=3, nr=4)
    ub, ib, _ = a.solve(w.rhs, rtol=1e-8)
    ref = _solver(w, precision="fp32_bf16", autotune=False)
    ur, ir, _ = ref.solve(w.rhs, rtol=1e-8)
    for u, i in ((ua, ia), (ub, ib)):
        assert (np.abs(i.astype(int) - ir.astype(int)) <= 2).all()
        assert np.linalg.norm(u - ur) <= 1e-6 * np.linalg.norm(ur)
    for bad in ({"bps_elem": 0}, {"bps_sub": 9}, {"depth": 7}, {"depth": -1}, {"nr": 3}, {"nr": 8},
                {"l2mode": 3}, {"l2keep": -1}):
        with pytest.raises(AmsError):
            a.set_launch_shape(3, **bad)
    with pytest.raises(AmsError):
        a.launch_shape(33)
    assert a.launch_shape(3)["depth"] == 3


def test_l2_priorities_leave_the_solve_bitwise_unchanged():
    """The L2 eviction priorities of the one-RHS local solve's tile copies
    change where the tiles are cached, not a single value: with the other
    shapes fixed, every priority setting gives the same bits."""
    w = make_small_2d(side=128, bs=32, m=4, std=2.0, seed=46)   # 32 block rows per subdomain
    s = _solver(w, precision="fp32_bf16", autotune=False)
    base = None
    for mode, keep in ((0, 0), (1, 0), (1, 3), (1, 1 << 20), (2, 3), (2, 1 << 20)):
        s.set_launch_shape(1, bps_elem=4, bps_sub=4, depth=2, nr=0, l2mode=mode, l2keep=keep)
        u, its, _ = s.solve(w.rhs[0], rtol=1e-8)
        if base is None:
            base = (u.copy(), its.copy())
        else:
            assert np.array_equal(u, base[0]) and np.array_equal(its, base[1]), (mode, keep)


def test_built_in_partition_when_none_is_given():
    """Without a partition the setup splits the pattern with ams_partition
    (seed 0, default imbalance): its subdomains are exactly that
    partition's parts, and PCG on them converges."""
    import scipy.sparse as sp
    from paper_2606_04864_gb300 import partition
    w = make_small_2d(side=96, bs=16, m=4, std=2.0, sigma=3.0, seed=47)
    part, _ = partition(w.rowptr, w.colind, 20)
    s = AmsSolver(w.rowptr, w.colind, w.vals, None, 20, 4, precision="fp32_bf16")
    perm, sub_ptr = s.index_maps()
    for i in range(20):
        assert np.array_equal(perm[sub_ptr[i]:sub_ptr[i + 1]], np.flatnonzero(part == i))
    u, its, rel = s.solve(w.rhs[0], rtol=1e-8)
    A = sp.csr_matrix((w.vals, w.colind, w.rowptr), shape=(w.n, w.n))
    assert rel[0] <= 1e-8
    assert np.linalg.norm(w.rhs[0] - A @ u) <= 1e-6 * np.linalg.norm(w.rhs[0])
    # a batch whose second system comes without a partition
    w2 = make_small_2d(side=40, bs=8, m=3, std=2.0, sigma=2.0, seed=48)
    b = AmsBatchedSolver([(w.rowptr, w.colind, w.vals, w.part, w.nparts, 4),
                          (w2.rowptr, w2.colind, w2.vals, None, 10, 3)], precision="fp32_bf16")
    ub, itb, relb = b.solve(b.pack([w.rhs[:1], w2.rhs[:1]]), 1, rtol=1e-8)
    u1, u2 = b.unpack(ub, 1)
    A2 = sp.csr_matrix((w2.vals, w2.colind, w2.rowptr), shape=(w2.n, w2.n))
    assert (relb <= 1e-8).all()
    assert np.linalg.norm(w2.rhs[0] - A2 @ u2[0]) <= 1e-6 * np.linalg.norm(w2.rhs[0])


def test_threshold_coarse_space_matches_oracle():
    """ams_options.eig_threshold: each subdomain keeps its local eigenvalues
    below the threshold (at least one, at most m); the counts equal the
    oracle's, subdomain by subdomain, and the FP64 solve matches the
    oracle's PCG on that coarse space."""
    w = make_small_2d(side=24, bs=6, m=8, std=2.0, sigma=3.0, seed=9)
    A = csr_to_scipy(w.rowptr, w.colind, w.vals)
    theta = 0.08
    o = OracleAMS(A, w.part, w.nparts, 8, eig_threshold=theta)
    near = np.concatenate([lam[:9] for lam in o.lams])
    assert np.min(np.abs(near - theta)) > 1e-3 * theta      # no count decided within rounding
    assert len(set(o.m_i)) > 1                              # the count does vary
    s = _solver(w, precision="fp64", eig_threshold=theta)
    mi, lam, psi = s.coarse_basis()
    assert mi.tolist() == list(o.m_i)
    ref = pcg(A, w.rhs[0], o.apply, rtol=1e-8)
    u, its, rel = s.solve(w.rhs[0], rtol=1e-8)
    assert abs(int(its[0]) - ref.iters) <= 2
    assert np.linalg.norm(u - ref.u) <= 1e-10 * np.linalg.norm(ref.u)
    with pytest.raises(AmsError):
        _solver(w, precision="fp64", eig_threshold=-1.0)


def test_profile_and_time_kernel_report_every_slot():
    """ams_profile_solve times every kernel slot of a real solve (one launch
    per slot and iteration, plus the first application), and ams_time_kernel
    times each slot on the solve state; both report the slot's algorithmic
    bytes."""
    from paper_2606_04864_gb300._lib import AMS_NUM_KERNELS, KERNEL_NAMES
    w = make_small_2d(side=64, bs=8, m=4, std=2.0, seed=44)
    s = _solver(w, precision="fp32_bf16")
    u, its, _ = s.solve(w.rhs[0], rtol=1e-8)
    prof = s.profile_solve(w.rhs[0], rtol=1e-8)
    assert [p["name"] for p in prof] == KERNEL_NAMES and len(prof) == AMS_NUM_KERNELS
    n_it = int(its[0])
    for k, p in enumerate(prof):
        # the direction slot runs once per iteration, the others also once for
        # z_0; iterations are launched in chunks, and launches after
        # convergence (at most one chunk of 64) return at once but are timed
        expect = n_it if k == 0 else n_it + 1
        assert expect <= p["count"] <= expect + 66, (p["name"], p["count"], expect)
        assert p["ms"] > 0 and p["bytes"] > 0
    for k in range(AMS_NUM_KERNELS):
        ms, by = s.time_kernel(k, 3)
        assert ms > 0 and by > 0


# ------------------------------------------------- many right-hand sides
# 16 and 32 right-hand sides take the code paths the one-to-six-RHS cases do
# not: local-solve warps whose right-hand-side group starts past 0 (several
# warps per block), the separate backward coarse substitution and the
# register-blocked coarse block products at 32 columns.

MANY = {
    "3d_b8": lambda nrhs: make_small_3d(side=16, bs=8, m=6, std=2.5, sigma=3.0, seed=32, nrhs=nrhs,
                                        rhs_kind="normal"),
    "2d_ragged": lambda nrhs: make_small_2d(side=45, bs=10, m=3, std=2.0, sigma=3.0, seed=31, ny=37,
                                            nrhs=nrhs, rhs_kind="normal"),
}


@pytest.fixture(scope="module", params=[(c, k) for c in MANY for k in (16, 32)],
                ids=lambda p: f"{p[0]}-{p[1]}rhs")
def many(request):
    name, nrhs = request.param
    w = MANY[name](nrhs)
    A = _A(w)
    o = OracleAMS(A, w.part, w.nparts, w.m)
    return name, nrhs, w, A, o


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 2e-5), ("fp32_bf16", 2e-5)])
def test_many_rhs_apply_matches_oracle(many, prec, tol):
    name, nrhs, w, A, o = many
    rnd = {"fp64": None, "fp32": "fp32", "fp32_bf16": "bf16"}[prec]
    orc = o if rnd is None else OracleAMS(A, w.part, w.nparts, w.m, basis_round=rnd)
    s = _solver(w, precision=prec)
    r = np.random.default_rng(7).standard_normal((nrhs, w.n))
    z = s.apply_preconditioner(r)
    for k in range(nrhs):
        zr = orc.apply(r[k])
        assert np.linalg.norm(z[k] - zr) <= tol * np.linalg.norm(zr), (prec, k)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_bf16"])
def test_many_rhs_pcg_matches_oracle(many, prec):
    """Every column: iterations within 2 of the oracle's PCG, solution within
    1e-10 (FP64 path) or max(1e-6, 10 x the oracle's own rtol-1e-8 error
    against its rtol-1e-13 solution) of the oracle."""
    name, nrhs, w, A, o = many
    s = _solver(w, precision=prec)
    u, its, rel = s.solve(w.rhs, rtol=1e-8)
    assert (rel <= 1e-8).all()
    for k in range(nrhs):
        ref = pcg(A, w.rhs[k], o.apply, rtol=1e-8)
        assert abs(int(its[k]) - ref.iters) <= 2, (k, its[k], ref.iters)
        err = np.linalg.norm(u[k] - ref.u) / np.linalg.norm(ref.u)
        if prec == "fp64":
            assert err <= 1e-10, (k, err)
        else:
            tight = pcg(A, w.rhs[k], o.apply, rtol=1e-13)
            floor = np.linalg.norm(ref.u - tight.u) / np.linalg.norm(tight.u)
            assert err <= max(1e-6, 10 * floor), (k, err, floor)


def test_autograd_solves_with_the_values_it_is_given():
    """ams_solve(vals, ...) loads vals into the solver before the forward:
    after log k changes, u and the gradient are those of the new matrix
    (the preconditioner is still the one built for the first matrix)."""
    from oracle import adjoint_gradient
    from paper_2606_04864_gb300.autograd import ams_solve
    from workloads import grf_logk, tpfa_csr, tpfa_values_from_logk
    w = make_small_3d(side=12, bs=4, m=4, std=2.0, sigma=2.0, seed=90)
    faces = w.extra["faces"]
    s = _solver(w, precision="fp64", device=True)
    f = torch.as_tensor(w.rhs[0], device="cuda")
    g_np = np.random.default_rng(91).standard_normal(w.n)
    for step, logk_np in enumerate([w.logk, w.logk + 0.7 * grf_logk(w.shape, 2.0, 1.0, 92)]):
        logk = torch.tensor(logk_np.reshape(-1), dtype=torch.float64, device="cuda", requires_grad=True)
        vals = tpfa_values_from_logk(logk, faces)
        vals.retain_grad()
        u = ams_solve(vals, f, s, rtol=1e-12)
        loss = torch.dot(u, torch.as_tensor(g_np, device="cuda"))
        loss.backward()
        rp, ci, vv = tpfa_csr(logk_np, faces)
        A = csr_to_scipy(rp, ci, vv)
        o = OracleAMS(A, w.part, w.nparts, w.m)
        ref = pcg(A, w.rhs[0], o.apply, rtol=1e-13)
        un = u.detach().cpu().numpy()
        assert np.linalg.norm(un - ref.u) <= 1e-9 * np.linalg.norm(ref.u), step
        lam_o, dv_o, _ = adjoint_gradient(A, ref.u, g_np, o.apply, rtol=1e-13)
        dv = vals.grad.detach().cpu().numpy()
        assert np.abs(dv - dv_o).max() <= 1e-8 * np.abs(dv_o).max(), step


def test_solve_into_a_caller_buffer():
    """solve(out=...) writes the solution into the caller's buffer (host:
    any C-contiguous float64 array, e.g. pinned memory; device: a CUDA
    tensor) and gives the same bits as the allocating call."""
    w = make_small_2d(side=40, bs=8, m=3, std=2.0, seed=93, nrhs=3, rhs_kind="normal")
    s = _solver(w, precision="fp32_bf16", autotune=False)
    u_ref, its_ref, _ = s.solve(w.rhs, rtol=1e-8)
    buf = torch.empty((3, w.n), dtype=torch.float64).pin_memory().numpy()
    u, its, _ = s.solve(w.rhs, rtol=1e-8, out=buf)
    assert u is buf and np.array_equal(buf, u_ref) and np.array_equal(its, its_ref)
    d = _solver(w, precision="fp32_bf16", autotune=False, device=True)
    tout = torch.empty((3, w.n), dtype=torch.float64, device="cuda")
    ud, _, _ = d.solve(torch.as_tensor(w.rhs, device="cuda"), rtol=1e-8, out=tout)
    assert ud is tout and np.array_equal(tout.cpu().numpy(), u_ref)
    with pytest.raises(ValueError):
        s.solve(w.rhs, rtol=1e-8, out=np.empty((2, w.n)))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32_bf16", 1e-6)])
def test_warm_start_matches_oracle_from_the_same_guess(prec, tol):
    """warm_start: CG from u_0 equals the oracle's CG from the same x_0
    (iterations within 2, solution within the path's tolerance); the exact
    solution as u_0 stops at k = 0; a zero right-hand side returns 0."""
    w = make_small_3d(side=16, bs=8, m=6, std=2.5, sigma=3.0, seed=32, nrhs=3, rhs_kind="normal")
    A = _A(w)
    o = OracleAMS(A, w.part, w.nparts, w.m)
    rng = np.random.default_rng(94)
    u0 = np.stack([np.linalg.solve(A.toarray(), w.rhs[k]) for k in range(3)])
    u0 = u0 + 1e-6 * rng.standard_normal(u0.shape) * np.abs(u0).max()
    f = w.rhs.copy()
    f[2] = 0.0
    s = _solver(w, precision=prec, warm_start=True)
    u, its, rel = s.solve(f, rtol=1e-8, u0=u0)
    flex = prec != "fp64"
    for k in range(2):
        ref = pcg(A, f[k], o.apply, rtol=1e-8, x0=u0[k], flexible=flex)
        cold = pcg(A, f[k], o.apply, rtol=1e-8, flexible=flex)
        assert abs(int(its[k]) - ref.iters) <= 2 and ref.iters < cold.iters, (k, its[k], ref.iters, cold.iters)
        assert np.linalg.norm(u[k] - ref.u) <= tol * np.linalg.norm(ref.u)
    assert its[2] == 0 and np.array_equal(u[2], np.zeros(w.n))
    exact = np.stack([np.linalg.solve(A.toarray(), f[k]) for k in range(3)])
    ue, itse, _ = s.solve(f[:2], rtol=1e-6, u0=exact[:2])
    assert (itse == 0).all() and np.array_equal(ue, exact[:2])
    with pytest.raises(ValueError):
        s.solve(f, rtol=1e-8)
