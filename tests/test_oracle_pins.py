"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed
forms, library routines that a special case reduces to, brute force on tiny
inputs, and the invariants of the paper's analysis (Section 4).  A mistake
anywhere in the oracle (a dropped term, a wrong sign or index, a transposed
operand) is meant to fail at least one of them; ``test_oracle_mutations``
plants a few such mistakes and checks that.
"""

import itertools

import numpy as np
import pytest
import scipy.linalg as la
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import (OracleAMS, adjoint_gradient, coarse_basis, coarse_matrix,
                    csr_to_scipy, index_maps, local_eigenpairs, local_matrices,
                    pcg)
from oracle.ams_oracle import local_eigenpairs_hep
from workloads import (block_partition, grf_logk, make_small_2d, make_small_3d,
                       tpfa_csr, tpfa_face_list)


def _A(w):
    return csr_to_scipy(w.rowptr, w.colind, w.vals)


# ---------------------------------------------------------------- index maps

def test_index_maps_brute_force():
    """Section 3.1: R_i selects the dofs of Omega_i; order is (part, index)."""
    rng = np.random.default_rng(0)
    for n, N in [(1, 1), (7, 3), (50, 6), (200, 17)]:
        part = rng.integers(0, N, size=n).astype(np.int32)
        part[:N if N <= n else n] = np.arange(min(N, n))   # no empty subdomain
        perm, iperm, sub_ptr = index_maps(part, N)
        expect = sorted(range(n), key=lambda g: (int(part[g]), g))
        assert perm.tolist() == expect
        assert (iperm[perm] == np.arange(n)).all()
        for i in range(N):
            assert (part[perm[sub_ptr[i]:sub_ptr[i + 1]]] == i).all()


def test_block_partition_ids():
    part, N = block_partition((6, 10), 4)   # 2 x 3 blocks, partial at the edges
    assert N == 6
    assert part.reshape(6, 10)[0, 0] == 0
    assert part.reshape(6, 10)[0, 9] == 2
    assert part.reshape(6, 10)[5, 0] == 3
    assert part.reshape(6, 10)[5, 9] == 5


# ------------------------------------------------------- TPFA test matrices

def test_tpfa_is_symmetric_m_matrix():
    for shape in [(9, 7), (5, 4, 6)]:
        logk = grf_logk(shape, 1.5, 2.0, 3)
        rowptr, colind, vals = tpfa_csr(logk)
        A = csr_to_scipy(rowptr, colind, vals)
        assert abs(A - A.T).max() == 0.0
        off = A - sp.diags(A.diagonal())
        assert off.max() <= 0.0
        assert (np.asarray(A.sum(axis=1)).ravel() > -1e-12 * A.diagonal().max()).all()
        # sorted columns in each row
        for i in range(A.shape[0]):
            c = colind[rowptr[i]:rowptr[i + 1]]
            assert (np.diff(c) > 0).all()
        np.linalg.cholesky(A.toarray())


def test_tpfa_uniform_is_five_point_laplacian():
    """Constant kappa = 1 on an s x s grid: interior rows are the 5-point
    stencil [-1, -1, 4, -1, -1]; a boundary face adds 2 to the diagonal."""
    s = 6
    rowptr, colind, vals = tpfa_csr(np.zeros((s, s)))
    A = csr_to_scipy(rowptr, colind, vals).toarray()
    i = 2 * s + 3
    assert A[i, i] == 4.0
    assert A[i, i - 1] == A[i, i + 1] == A[i, i - s] == A[i, i + s] == -1.0
    assert A[0, 0] == 2.0 + 2.0 + 2.0     # two inner faces + two wall faces


# -------------------------------------------------- local matrices, Sec. 3.2

def test_local_matrix_definitions_brute_force():
    w = make_small_2d(side=6, bs=3, m=2, std=1.5, seed=4)
    A = _A(w).toarray()
    perm, iperm, sub_ptr = index_maps(w.part, w.nparts)
    for i in range(w.nparts):
        dofs = perm[sub_ptr[i]:sub_ptr[i + 1]]
        Ai, Ahat, s = local_matrices(_A(w), dofs)
        for a, b in itertools.product(range(len(dofs)), repeat=2):
            assert Ai[a, b] == A[dofs[a], dofs[b]]
            if a != b:
                assert Ahat[a, b] == A[dofs[a], dofs[b]]
        for a in range(len(dofs)):
            off = sum(A[dofs[a], dofs[b]] for b in range(len(dofs)) if b != a)
            assert abs(Ahat[a, a] + off) <= 1e-15 * abs(off)
            assert s[a] == Ahat[a, a]
        assert np.abs(Ahat.sum(axis=1)).max() <= 1e-12 * s.max()
        assert np.linalg.eigvalsh(Ahat).min() >= -1e-12 * s.max()


def test_isolated_dof_weight_reading():
    """A dof with no in-subdomain neighbour has S_jj = 0; the reading sets
    S_jj = A_jj, which gives it an eigenvalue 0 of its own."""
    w = make_small_2d(side=4, bs=4, m=2, seed=1)
    A = _A(w)
    dofs = np.array([0, 5, 10])              # diagonal cells: no mutual faces
    Ai, Ahat, s = local_matrices(A, dofs)
    assert (np.diag(Ahat) == 0).all()
    assert (s == A.diagonal()[dofs]).all()
    lam, Psi, mi = local_eigenpairs(Ahat, s, 2)
    assert np.allclose(lam, 0.0)


# ---------------------------------------------------------- eigenpairs

def test_eigenpairs_residual_and_s_orthonormality():
    w = make_small_3d(side=8, bs=4, m=5, std=2.0, seed=2)
    o = OracleAMS(_A(w), w.part, w.nparts, w.m)
    for i, dofs in enumerate(o.sub_dofs):
        Ai, Ahat, s = local_matrices(o.A, dofs)
        Psi = o.Psis[i]
        lam = o.lams[i][:Psi.shape[1]]
        R = Ahat @ Psi - (s[:, None] * Psi) * lam[None, :]
        assert np.abs(R).max() <= 1e-12 * np.abs(Ahat).max()
        G = Psi.T @ (s[:, None] * Psi)
        assert np.abs(G - np.eye(Psi.shape[1])).max() <= 1e-12


def test_first_mode_is_constant():
    """Zero row sums: the constant vector spans the kernel of \\hat A_i on a
    connected subdomain, so lambda_1 = 0 and psi_1 = 1/sqrt(sum_j S_jj)."""
    w = make_small_2d(side=12, bs=4, m=3, std=2.0, seed=7)
    o = OracleAMS(_A(w), w.part, w.nparts, w.m)
    for i, dofs in enumerate(o.sub_dofs):
        Ai, Ahat, s = local_matrices(o.A, dofs)
        assert abs(o.lams[i][0]) <= 1e-13
        psi1 = o.Psis[i][:, 0]
        expect = 1.0 / np.sqrt(s.sum())
        assert np.abs(psi1 - expect).max() <= 1e-12 * expect


@pytest.mark.parametrize("n", [2, 3, 9, 20])
def test_path_subdomain_closed_form(n):
    """A 1-D chain of n cells with uniform coupling: \\hat A is the path
    Laplacian and S its degree matrix, whose generalized eigenvalues are
    lambda_k = 1 - cos(pi k/(n-1)), k = 0..n-1 (random-walk Laplacian of a
    path)."""
    logk = np.zeros((1, n))
    rowptr, colind, vals = tpfa_csr(logk)
    A = csr_to_scipy(rowptr, colind, vals)
    Ai, Ahat, s = local_matrices(A, np.arange(n))
    lam, Psi, mi = local_eigenpairs(Ahat, s, n)
    expect = 1.0 - np.cos(np.pi * np.arange(n) / (n - 1))
    assert np.abs(lam - expect).max() <= 1e-13


def test_ghep_and_hep_have_the_same_spectrum():
    """Section 5.3: S^{-1/2} \\hat A S^{-1/2} has the spectrum of the pencil
    and psi = S^{-1/2} z spans the same eigenspaces."""
    w = make_small_2d(side=10, bs=5, m=4, std=2.5, seed=9)
    A = _A(w)
    perm, iperm, sub_ptr = index_maps(w.part, w.nparts)
    for i in range(w.nparts):
        dofs = perm[sub_ptr[i]:sub_ptr[i + 1]]
        Ai, Ahat, s = local_matrices(A, dofs)
        lam_g, Psi_g, mi = local_eigenpairs(Ahat, s, 4)
        lam_h, Psi_h = local_eigenpairs_hep(Ahat, s, 4)
        assert np.abs(lam_g - lam_h).max() <= 1e-13
        Pg = Psi_g @ Psi_g.T @ np.diag(s)
        Ph = Psi_h @ Psi_h.T @ np.diag(s)
        assert np.abs(Pg - Ph).max() <= 1e-10


def test_cluster_at_cut_is_closed():
    """A uniform square block has a D4 symmetry: the modes (1,0)/(0,1) are
    a double eigenvalue, so m = 2 would split it; the oracle grows m_i to 3."""
    w = make_small_2d(side=8, bs=8, m=2, std=0.0, seed=0)
    A = _A(w)
    Ai, Ahat, s = local_matrices(A, np.arange(w.n))
    lam, Psi, mi = local_eigenpairs(Ahat, s, 2)
    assert abs(lam[1] - lam[2]) <= 1e-10 * lam[2]
    assert mi == 3


# ------------------------------------------------------- coarse space

def test_full_coarse_space_reproduces_inverse():
    """Keeping every local mode makes R_0^T square and invertible, so
    R_0^T A_0^{-1} R_0 = A^{-1}; with the additive form,
    M^{-1} - sum_i R_i^T A_i^{-1} R_i = A^{-1}."""
    w = make_small_2d(side=8, bs=4, m=16, std=2.0, seed=11)
    A = _A(w)
    o = OracleAMS(A, w.part, w.nparts, w.m)
    assert o.Nc == w.n
    Ainv = np.linalg.inv(A.toarray())
    C = np.column_stack([o.coarse_part(e) for e in np.eye(w.n)])
    assert np.abs(C - Ainv).max() <= 1e-10 * np.abs(Ainv).max()
    # coarse-only preconditioner: PCG converges in one iteration
    res = pcg(A, w.rhs[0], o.coarse_part, rtol=1e-10)
    assert res.iters == 1


def test_coarse_matrix_spd_and_galerkin_brute_force():
    w = make_small_2d(side=8, bs=4, m=3, std=2.0, seed=12)
    A = _A(w)
    o = OracleAMS(A, w.part, w.nparts, w.m)
    A0 = o.A0
    R = o.R0T.toarray()
    assert np.abs(A0 - R.T @ A.toarray() @ R).max() <= 1e-12 * np.abs(A0).max()
    assert np.abs(A0 - A0.T).max() <= 1e-14 * np.abs(A0).max()
    assert np.linalg.eigvalsh(A0).min() > 0


def test_one_mode_is_unsmoothed_aggregation():
    """m = 1 on connected subdomains: psi_1 is constant, so R_0^T is the
    aggregation (piecewise-constant) prolongator with S-normalised columns."""
    w = make_small_2d(side=8, bs=4, m=1, std=2.0, seed=13)
    A = _A(w)
    o = OracleAMS(A, w.part, w.nparts, w.m)
    R = o.R0T.toarray()
    for i, dofs in enumerate(o.sub_dofs):
        col = R[:, i]
        assert np.count_nonzero(col) == len(dofs)
        assert np.ptp(col[dofs]) <= 1e-13 * col[dofs].max()


def test_preconditioner_symmetric_positive_definite():
    w = make_small_2d(side=8, bs=4, m=2, std=2.0, seed=14)
    o = OracleAMS(_A(w), w.part, w.nparts, w.m)
    M = o.dense_Minv()
    assert np.abs(M - M.T).max() <= 1e-12 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


# ------------------------------------------------------------ PCG

def test_pcg_solution_matches_dense_cholesky():
    w = make_small_2d(side=16, bs=4, m=3, std=2.0, seed=15)
    A = _A(w)
    o = OracleAMS(A, w.part, w.nparts, w.m)
    f = w.rhs[0]
    u_ref = la.cho_solve(la.cho_factor(A.toarray()), f)
    res = pcg(A, f, o.apply, rtol=1e-12)
    assert res.converged
    assert np.linalg.norm(res.u - u_ref) <= 1e-10 * np.linalg.norm(u_ref)
    assert res.true_relres <= 1e-11


def test_block_jacobi_special_case_matches_scipy_cg():
    """m = 0: the preconditioner is block Jacobi; scipy's CG with the same
    operator takes the same iterations and reaches the same solution."""
    w = make_small_2d(side=16, bs=4, m=0, std=2.0, seed=16)
    A = _A(w)
    o = OracleAMS(A, w.part, w.nparts, 0, coarse=False)
    f = w.rhs[0]
    res = pcg(A, f, o.apply, rtol=1e-8)
    it = [0]

    def cb(xk):
        it[0] += 1

    M = spla.LinearOperator(A.shape, matvec=o.apply)
    x, info = spla.cg(A, f, rtol=1e-8, atol=0.0, M=M, maxiter=1000, callback=cb)
    assert info == 0
    assert abs(it[0] - res.iters) <= 1
    assert np.linalg.norm(x - res.u) <= 1e-7 * np.linalg.norm(x)


def test_single_subdomain_converges_in_one_iteration():
    w = make_small_2d(side=8, bs=8, m=2, std=2.0, seed=17)
    A = _A(w)
    o = OracleAMS(A, w.part, w.nparts, w.m)
    assert w.nparts == 1
    res = pcg(A, w.rhs[0], o.local_part, rtol=1e-10)
    assert res.iters == 1


def test_flexible_cg_equals_pcg_for_symmetric_preconditioner():
    w = make_small_2d(side=16, bs=4, m=2, std=2.0, seed=18)
    A = _A(w)
    o = OracleAMS(A, w.part, w.nparts, w.m)
    a = pcg(A, w.rhs[0], o.apply, rtol=1e-8)
    b = pcg(A, w.rhs[0], o.apply, rtol=1e-8, flexible=True)
    assert a.iters == b.iters
    assert np.linalg.norm(a.u - b.u) <= 1e-9 * np.linalg.norm(a.u)


def test_lanczos_ritz_values_match_dense_spectrum():
    """CG's alpha/beta define the Lanczos tridiagonal of M^{-1}A; its
    extreme Ritz values converge to the extreme eigenvalues of M^{-1}A."""
    w = make_small_2d(side=12, bs=4, m=2, std=2.0, seed=19)
    A = _A(w)
    o = OracleAMS(A, w.part, w.nparts, w.m)
    res = pcg(A, w.rhs[0], o.apply, rtol=1e-14, maxit=200)
    a, b = res.alphas, res.betas
    k = min(len(a), len(b) + 1)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / a[j] + (b[j - 1] / a[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(b[j]) / a[j]
    ritz = np.linalg.eigvalsh(T)
    ev = np.sort(np.linalg.eigvals(o.dense_Minv() @ A.toarray()).real)
    assert abs(ritz[-1] - ev[-1]) <= 1e-6 * ev[-1]
    assert abs(ritz[0] - ev[0]) <= 1e-6 * ev[0]


def test_iterations_do_not_grow_with_more_modes():
    """Section 5.3: a richer coarse space lowers the iteration count."""
    w = make_small_2d(side=32, bs=8, m=1, std=2.5, seed=20)
    A = _A(w)
    its = []
    for m in (1, 3, 6, 10):
        o = OracleAMS(A, w.part, w.nparts, m)
        its.append(pcg(A, w.rhs[0], o.apply, rtol=1e-8).iters)
    assert all(its[j + 1] <= its[j] + 1 for j in range(len(its) - 1)), its
    assert its[-1] < its[0]


# ----------------------------------------------- analysis invariants (Sec 4)

def _random_vectors(n, k, seed):
    return np.random.default_rng(seed).standard_normal((k, n))


def test_lemma1_s_norm_is_additive():
    w = make_small_2d(side=12, bs=4, m=2, std=2.0, seed=21)
    A = _A(w)
    o = OracleAMS(A, w.part, w.nparts, w.m)
    svec = np.zeros(w.n)
    locs = []
    for dofs in o.sub_dofs:
        Ai, Ahat, s = local_matrices(A, dofs)
        svec[dofs] = s
        locs.append((dofs, s))
    for x in _random_vectors(w.n, 5, 1):
        lhs = x @ (svec * x)
        rhs = sum(x[d] @ (s * x[d]) for d, s in locs)
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_lemma2_local_energy_below_global_energy():
    w = make_small_3d(side=8, bs=4, m=2, std=2.0, seed=22)
    A = _A(w)
    perm, iperm, sub_ptr = index_maps(w.part, w.nparts)
    for x in _random_vectors(w.n, 10, 2):
        glob = x @ (A @ x)
        loc = 0.0
        for i in range(w.nparts):
            d = perm[sub_ptr[i]:sub_ptr[i + 1]]
            Ai, Ahat, s = local_matrices(A, d)
            loc += x[d] @ (Ahat @ x[d])
        assert loc <= glob * (1 + 1e-12)


def test_theorem2_local_approximation_bound():
    """||x_i - Pi_i x_i||_S^2 <= ||x_i||_Ahat^2 / lambda_{m_i+1}."""
    w = make_small_2d(side=12, bs=6, m=3, std=2.0, seed=23)
    A = _A(w)
    o = OracleAMS(A, w.part, w.nparts, w.m)
    for i, dofs in enumerate(o.sub_dofs):
        Ai, Ahat, s = local_matrices(A, dofs)
        Psi = o.Psis[i]
        lam_next = o.lams[i][Psi.shape[1]]
        for x in _random_vectors(len(dofs), 5, 3 + i):
            Pix = Psi @ (Psi.T @ (s * x))
            e = x - Pix
            assert e @ (s * e) <= (x @ (Ahat @ x)) / lam_next * (1 + 1e-10)


def test_theorem1_bound_tight_at_optimal_scaling():
    """With P^{-1} = omega M^{-1}, omega = 2/(l_min + l_max), the A-norm of
    E = I - P^{-1}A is delta = (l_max - l_min)/(l_max + l_min) < 1 and
    Theorem 1's bound (1+delta)/(1-delta) equals kappa(M^{-1}A)."""
    w = make_small_2d(side=8, bs=4, m=2, std=2.0, seed=24)
    A = _A(w).toarray()
    o = OracleAMS(_A(w), w.part, w.nparts, w.m)
    M = o.dense_Minv()
    ev = np.sort(np.linalg.eigvals(M @ A).real)
    omega = 2.0 / (ev[0] + ev[-1])
    E = np.eye(w.n) - omega * M @ A
    L = np.linalg.cholesky(A)
    EA = L.T @ E @ np.linalg.inv(L.T)         # A-norm = 2-norm of A^{1/2} E A^{-1/2}
    delta = np.linalg.norm(EA, 2)
    assert delta < 1
    kappa = ev[-1] / ev[0]
    assert kappa <= (1 + delta) / (1 - delta) * (1 + 1e-8)
    assert abs(kappa - (1 + delta) / (1 - delta)) <= 1e-6 * kappa


# ------------------------------------------------------------ adjoint

def test_adjoint_matches_dense_and_closed_form_and_fd():
    """dL/dA_ij = -lambda_i u_j; chained to a face transmissibility T_f
    between cells i, j this is -(lambda_i - lambda_j)(u_i - u_j), and for a
    wall face -lambda_i u_i.  Checked against dense solves, the closed
    form, and central differences of L(kappa) = 0.5 ||u[obs] - d||^2."""
    w = make_small_2d(side=6, bs=3, m=2, std=1.0, seed=25)
    faces = w.extra["faces"]
    A = _A(w)
    f = w.rhs[0]
    o = OracleAMS(A, w.part, w.nparts, w.m)
    obs = np.array([3, 10, 17, 30])
    d = np.linspace(0.0, 1e-3, len(obs))

    def loss_of(logk):
        rp, ci, v = tpfa_csr(logk.reshape(w.shape), faces)
        Ad = csr_to_scipy(rp, ci, v).toarray()
        u = np.linalg.solve(Ad, f)
        return 0.5 * np.sum((u[obs] - d) ** 2), u

    L0, u_dense = loss_of(w.logk.reshape(-1))
    u = pcg(A, f, o.apply, rtol=1e-13).u
    assert np.linalg.norm(u - u_dense) <= 1e-11 * np.linalg.norm(u_dense)
    g = np.zeros(w.n)
    g[obs] = u[obs] - d
    lam, dvals, res = adjoint_gradient(A, u, g, o.apply, rtol=1e-13)
    lam_dense = np.linalg.solve(A.toarray(), g)
    assert np.linalg.norm(lam - lam_dense) <= 1e-10 * np.linalg.norm(lam_dense)
    # face closed form
    # A_ij = A_ji = -T and T is added to A_ii and A_jj
    dT = -dvals[faces.pos_ij] - dvals[faces.pos_ji] + dvals[faces.pos_ii] + dvals[faces.pos_jj]
    closed = -(lam[faces.fi] - lam[faces.fj]) * (u[faces.fi] - u[faces.fj])
    assert np.abs(dT - closed).max() <= 1e-12 * np.abs(closed).max()
    dTb = np.zeros(len(faces.bcell))
    dTb[:] = dvals[faces.pos_b]
    assert np.abs(dTb + lam[faces.bcell] * u[faces.bcell]).max() <= 1e-12 * np.abs(dTb).max()
    # chain to log k and compare with central differences
    k = np.exp(w.logk.reshape(-1))
    ki, kj = k[faces.fi], k[faces.fj]
    dlogk = np.zeros(w.n)
    np.add.at(dlogk, faces.fi, dT * faces.hfac * 2 * kj ** 2 / (ki + kj) ** 2 * ki)
    np.add.at(dlogk, faces.fj, dT * faces.hfac * 2 * ki ** 2 / (ki + kj) ** 2 * kj)
    np.add.at(dlogk, faces.bcell, dTb * faces.hfac * 2 * k[faces.bcell])
    rng = np.random.default_rng(5)
    h = 1e-6
    for _ in range(4):
        v = rng.standard_normal(w.n)
        lp, _ = loss_of(w.logk.reshape(-1) + h * v)
        lm, _ = loss_of(w.logk.reshape(-1) - h * v)
        fd = (lp - lm) / (2 * h)
        an = dlogk @ v
        assert abs(fd - an) <= 1e-5 * max(abs(an), 1e-30)


# ------------------------------------------------- multiplicative two-grid cycle

def _dense(op, n):
    return np.column_stack([op(e) for e in np.eye(n)])


def _two_grid_case(m=3, seed=5):
    w = make_small_2d(side=24, bs=6, m=m, std=2.0, sigma=3.0, seed=seed)
    A = _A(w)
    return w, A, OracleAMS(A, w.part, w.nparts, w.m)


def test_two_grid_cycle_is_symmetric_positive_definite():
    """Pre- and post-smoothing with the same symmetric smoother make the
    cycle symmetric; with a convergent smoother (omega < 2/lambda_max(SA))
    and an exact coarse solve, the spectrum of B A lies in (0, 1]."""
    w, A, o = _two_grid_case()
    lmax = o.local_lambda_max()
    Ad = A.toarray()
    Sd = _dense(o.local_part, o.n)
    exact = la.eigvals(Sd @ Ad).real.max()
    assert exact * (1 - 1e-6) <= lmax <= exact * (1 + 1e-12)
    for omega in (0.5 / lmax, 1.0 / lmax, 1.9 / lmax):
        B = _dense(lambda r: o.apply_two_grid(r, omega), o.n)
        assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
        ev = la.eigvals(B @ Ad).real
        assert ev.min() > 0 and ev.max() <= 1 + 1e-10


def test_two_grid_full_coarse_space_is_the_inverse():
    """Keeping every local mode makes the coarse correction exact: the
    error after it is zero and post-smoothing keeps it zero, so B = A^{-1}
    for any omega."""
    w = make_small_2d(side=12, bs=4, m=16, std=2.0, seed=21)
    A = _A(w)
    o = OracleAMS(A, w.part, w.nparts, 16)
    assert o.Nc == o.n
    Ainv = la.inv(A.toarray())
    for omega in (0.3, 0.7, 1.0):
        B = _dense(lambda r: o.apply_two_grid(r, omega), o.n)
        assert np.abs(B - Ainv).max() <= 1e-9 * np.abs(Ainv).max()


def test_two_grid_without_coarse_space_is_the_symmetrised_smoother():
    """With no coarse space the cycle is two smoothing steps,
    B = 2 omega S - omega^2 S A S (S the sum of local solves)."""
    w = make_small_2d(side=16, bs=4, m=2, std=2.0, seed=22)
    A = _A(w)
    o = OracleAMS(A, w.part, w.nparts, 0, coarse=False)
    Sd = _dense(o.local_part, o.n)
    Ad = A.toarray()
    omega = 0.6
    B = _dense(lambda r: o.apply_two_grid(r, omega), o.n)
    ref = 2 * omega * Sd - omega ** 2 * Sd @ Ad @ Sd
    assert np.abs(B - ref).max() <= 1e-12 * np.abs(ref).max()


def _rbar_and_error(o, A, omega):
    Ad = A.toarray()
    Sd = _dense(o.local_part, o.n)
    Rbar = 2 * omega * Sd - omega ** 2 * Sd @ Ad @ Sd       # symmetrised smoother
    B = _dense(lambda r: o.apply_two_grid(r, omega), o.n)
    E = np.eye(o.n) - B @ Ad                                # error propagation
    normE = la.eigvals(E).real.max()                        # E is A-self-adjoint, >= 0
    return Ad, Rbar, normE


def test_two_grid_identity_of_the_abstract_theory():
    """The two-grid identity the Analysis (Section 4) builds on:
    ||E||_A = 1 - 1/K with K = max_v min_{v_c} ||v - v_c||^2_{Rbar^{-1}} /
    ||v||_A^2 over the coarse space, Rbar the symmetrised smoother.  K is
    computed here from a generalised eigenproblem, independently of the
    cycle."""
    for m, seed in ((2, 5), (4, 6)):
        w, A, o = _two_grid_case(m=m, seed=seed)
        omega = 1.0 / o.local_lambda_max()
        Ad, Rbar, normE = _rbar_and_error(o, A, omega)
        W = la.inv(Rbar)
        P = o.R0T.toarray()
        proj = P @ la.solve(P.T @ W @ P, P.T @ W)          # W-orthogonal projection onto range(P)
        Q = np.eye(o.n) - proj
        K = la.eigh(Q.T @ W @ Q, Ad, eigvals_only=True).max()
        assert abs(normE - (1 - 1 / K)) <= 1e-8


def test_two_grid_bound_of_the_convergence_theorem():
    """Section 4: ||E||_A <= 1 - mu_c / C, where mu_c = min_i lambda^(i)_{m_i+1}
    (the first local eigenvalue left out of the coarse space) and C bounds
    the symmetrised smoother against the weighting matrix,
    ||v||^2_{Rbar^{-1}} <= C ||v||^2_S."""
    w, A, o = _two_grid_case(m=3, seed=7)
    omega = 1.0 / o.local_lambda_max()
    Ad, Rbar, normE = _rbar_and_error(o, A, omega)
    s = np.zeros(o.n)
    for dofs in o.sub_dofs:
        s[dofs] = local_matrices(A, dofs)[2]
    d = 1 / np.sqrt(s)
    C = la.eigh(d[:, None] * la.inv(Rbar) * d[None, :], eigvals_only=True).max()
    mu_c = min(lam[Psi.shape[1]] for lam, Psi in zip(o.lams, o.Psis))
    assert 0 < normE <= 1 - mu_c / C + 1e-12


def test_two_grid_pcg_reaches_the_dense_solution():
    w, A, o = _two_grid_case()
    omega = 1.0 / o.local_lambda_max()
    res = pcg(A, w.rhs[0], lambda r: o.apply_two_grid(r, omega), rtol=1e-10)
    u = la.solve(A.toarray(), w.rhs[0], assume_a="pos")
    assert res.converged
    assert np.linalg.norm(res.u - u) <= 1e-8 * np.linalg.norm(u)


# ------------------------------------------------ adaptive m_i by threshold

def test_threshold_count_and_the_bound_it_buys():
    """m_i = the local eigenvalues below the threshold (at least one, at most
    m, grown across a cluster): every kept eigenvalue is below it except the
    floor's single mode, the first left out is at or above it unless the cap
    binds, so mu_c >= threshold; with the two-grid cycle the Section 4 bound
    then gives ||E||_A <= 1 - threshold / C."""
    w = make_small_2d(side=24, bs=6, m=8, std=2.0, sigma=3.0, seed=9)
    A = _A(w)
    theta = 0.08
    o = OracleAMS(A, w.part, w.nparts, 8, eig_threshold=theta)
    capped = 0
    for dofs, lam, Psi in zip(o.sub_dofs, o.lams, o.Psis):
        Ai, Ahat, s = local_matrices(A, dofs)
        ref = la.eigh(Ahat, np.diag(s), eigvals_only=True)      # independent count
        mi = Psi.shape[1]
        below = int(np.count_nonzero(ref < theta))
        assert mi == min(max(below, 1), 8) or (mi > min(max(below, 1), 8) and
                                                abs(ref[mi - 1] - ref[mi - 2]) <= 1e-8 * abs(ref[mi - 1]))
        if mi < 8:
            assert ref[mi] >= theta
        else:
            capped += 1
    assert capped < len(o.sub_dofs)
    if capped == 0:
        omega = 1.0 / o.local_lambda_max()
        Ad, Rbar, normE = _rbar_and_error(o, A, omega)
        sw = np.zeros(o.n)
        for dofs in o.sub_dofs:
            sw[dofs] = local_matrices(A, dofs)[2]
        d = 1 / np.sqrt(sw)
        C = la.eigh(d[:, None] * la.inv(Rbar) * d[None, :], eigvals_only=True).max()
        assert normE <= 1 - theta / C + 1e-12


def test_higher_threshold_keeps_more_modes_and_no_more_iterations():
    w = make_small_2d(side=24, bs=6, m=8, std=2.0, sigma=3.0, seed=9)
    A = _A(w)
    prev_m, prev_it = -1, 10 ** 9
    for theta in (0.02, 0.08, 0.3):
        o = OracleAMS(A, w.part, w.nparts, 8, eig_threshold=theta)
        res = pcg(A, w.rhs[0], o.apply, rtol=1e-10)
        assert o.Nc >= prev_m and res.iters <= prev_it + 1
        prev_m, prev_it = o.Nc, res.iters


# ------------------------------------------------ reduced-precision basis storage
# The mixed-precision parity tests compare the GPU with an oracle whose basis
# is rounded the way the GPU stores it (round_basis), so the rounding itself
# is pinned here against hand-worked values of the formats and two
# independent converters.

_BF16_CASES = [
    # (input, bfloat16 value): 8 significant bits, round to nearest, ties to even
    (1.0, 1.0),
    (1.0 + 2.0 ** -9, 1.0),                              # below half a spacing (2^-7)
    (1.0 + 2.0 ** -8, 1.0),                              # tie, 1.0 is even
    (1.0 + 3 * 2.0 ** -9, 1.0 + 2.0 ** -7),              # above half
    (1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -6),              # tie, 1+2^-7 is odd: up
    (1.0 + 2.0 ** -8 + 2.0 ** -40, 1.0 + 2.0 ** -7),     # just above a tie: rounded from FP64 directly
    (2.0 - 2.0 ** -9, 2.0),                              # carry into the exponent
    (2.0 - 2.0 ** -8, 2.0),                              # tie, 2 - 2^-7 is odd: up to 2
    (-(1.0 + 3 * 2.0 ** -9), -(1.0 + 2.0 ** -7)),        # sign symmetric
    (0.3, 0.30078125),                                   # 0.3 = 1.2 * 2^-2 -> 154/128 * 2^-2
    (-0.0, -0.0),
    (0.0, 0.0),
    (2.0 ** -130 + 2.0 ** -134, 2.0 ** -130),            # subnormal tie (8.5 spacings of 2^-133): even
    (2.0 ** -130 + 3 * 2.0 ** -134, 5 * 2.0 ** -132),    # subnormal tie (9.5 spacings): up to 10
    (2.0 ** -135, 0.0),                                  # a quarter spacing
    (3 * 2.0 ** -135, 2.0 ** -133),                      # three quarters: the smallest subnormal
    ((2 - 2.0 ** -7) * 2.0 ** 127, (2 - 2.0 ** -7) * 2.0 ** 127),   # largest finite value
    ((2 - 2.0 ** -8) * 2.0 ** 127, np.inf),              # tie above it rounds to 2^128: overflow
]


def test_bf16_rounding_hand_worked_values():
    from oracle.ams_oracle import round_basis
    x = np.array([c[0] for c in _BF16_CASES])
    want = np.array([c[1] for c in _BF16_CASES])
    got = round_basis(x, "bf16")
    assert np.array_equal(got, want), [(a, b, c) for a, b, c in zip(x, got, want) if b != c]
    assert np.array_equal(np.signbit(got), np.signbit(want))


def _bf16_rne_from_binary32_bits(x32: np.ndarray) -> np.ndarray:
    """Textbook integer rounding of binary32 bit patterns to their upper 16
    bits (add 0x7FFF plus the lowest kept bit, drop 16 bits); exact for
    finite binary32 inputs, subnormals included."""
    b = x32.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_rounding_matches_integer_rounding_and_torch_on_binary32_inputs():
    """On values that binary32 holds exactly, FP64 -> bfloat16 and
    binary32 -> bfloat16 are the same rounding, so two independent
    converters apply: the integer bit trick and torch's bfloat16 cast."""
    import torch
    from oracle.ams_oracle import round_basis
    rng = np.random.default_rng(5)
    parts = [rng.standard_normal(20000),
             rng.uniform(-1, 1, 20000) * 2.0 ** rng.integers(-140, 120, 20000),   # wide exponents, subnormals
             (1.0 + np.arange(512) * 2.0 ** -16) * rng.choice([-1.0, 1.0], 512)]  # every tie pattern near 1
    x32 = np.concatenate(parts).astype(np.float32)
    x32 = x32[np.isfinite(x32)]
    x = x32.astype(np.float64)
    got = round_basis(x, "bf16")
    assert np.array_equal(got, _bf16_rne_from_binary32_bits(x32))
    via_torch = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(got, via_torch)


def test_fp32_rounding_matches_binary32():
    from oracle.ams_oracle import round_basis
    rng = np.random.default_rng(6)
    x = rng.standard_normal(1000) * 2.0 ** rng.integers(-160, 120, 1000)
    got = round_basis(x, "fp32")
    # binary32 keeps 24 significant bits: |x - fl(x)| <= 2^-24 |x| for normals
    normal = np.abs(x) >= 2.0 ** -126
    assert np.all(np.abs(got - x)[normal] <= 2.0 ** -24 * np.abs(x[normal]))
    assert round_basis(np.array([1.0 + 2.0 ** -24]), "fp32")[0] == 1.0          # tie to even
    assert round_basis(np.array([1.0 + 3 * 2.0 ** -24]), "fp32")[0] == 1.0 + 2.0 ** -22


def test_pcg_from_an_initial_guess():
    """CG from x_0: the exact solution as x_0 stops at once (k = 0), x_0 = 0
    reproduces the default path bit for bit, and any x_0 converges to the
    dense solution at the requested relative residual of f."""
    w = make_small_2d(side=20, bs=5, m=3, std=2.0, seed=17)
    A = _A(w)
    o = OracleAMS(A, w.part, w.nparts, w.m)
    f = w.rhs[0]
    u_exact = np.linalg.solve(A.toarray(), f)
    r0 = pcg(A, f, o.apply, rtol=1e-8, x0=u_exact)
    assert r0.iters == 0 and np.array_equal(r0.u, u_exact)
    base = pcg(A, f, o.apply, rtol=1e-8)
    zero = pcg(A, f, o.apply, rtol=1e-8, x0=np.zeros_like(f))
    assert zero.iters == base.iters and np.array_equal(zero.u, base.u)
    x0 = np.random.default_rng(4).standard_normal(w.n)
    res = pcg(A, f, o.apply, rtol=1e-10, x0=x0)
    assert res.converged and np.linalg.norm(f - A @ res.u) <= 2e-10 * np.linalg.norm(f)
    assert np.linalg.norm(res.u - u_exact) <= 1e-7 * np.linalg.norm(u_exact)
    # a good initial guess saves iterations
    near = pcg(A, f, o.apply, rtol=1e-8, x0=u_exact + 1e-6 * x0)
    assert near.iters < base.iters
    # f = 0: the solution is 0 whatever x_0 is
    assert np.array_equal(pcg(A, np.zeros(w.n), o.apply, x0=x0).u, np.zeros(w.n))
