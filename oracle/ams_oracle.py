"""Plain FP64 oracle of the AMS-preconditioned CG solve (test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline/reference legs, never by the library.  It
shares no code with the CUDA path; the only common inputs are the seeded
matrices from ``workloads``.

Every step follows the paper (arXiv 2606.04864, "An algebraic multiscale
preconditioner for large sparse SPD matrices") in its own order and notation:

* Section 3.1: non-overlapping subdomains Omega_i from a graph partition,
  prolongation R_0^T, Galerkin coarse matrix A_0 = R_0 A R_0^T, two-level
  preconditioner built around R_0^T A_0^+ R_0.
* Section 3.2: A_i = R_i A R_i^T; \\hat A_i = A_i with each diagonal entry
  replaced by minus the sum of the row's off-diagonal entries (zero row
  sums); S_i = diag(\\hat A_i); the generalized eigenproblem
  \\hat A_i psi = lambda S_i psi (Eq. algebraic-eigenproblem); the m_i
  eigenvectors of smallest eigenvalue, zero-extended and concatenated
  subdomain by subdomain, are the columns of R_0^T.
* Section 5 (experimental setup): the equivalent standard problem
  S^{-1/2} \\hat A S^{-1/2} z = lambda z with psi = S^{-1/2} z.

Readings where the paper is silent (each is listed in the design notes):

* Preconditioner form: additive two-level,
  M^{-1} = sum_i R_i^T A_i^{-1} R_i + R_0^T A_0^{-1} R_0.  The paper's
  printed P^{-1} = R_0^T A_0^+ R_0 is singular on its own; its convergence
  theorem (Theorem 2) has a smoother constant C, so a fine-level component
  is implied.  The fine-level component uses the Dirichlet-type A_i (SPD),
  not the singular \\hat A_i.
* A_0 is SPD for the Dirichlet test matrices, so A_0^+ = A_0^{-1} and a
  Cholesky factorisation is used; a non-positive pivot is an error.
* A zero S_jj (a dof with no in-subdomain neighbour) is replaced by A_jj.
* m_i = min(m, n_i); if lambda_{m_i+1} equals lambda_{m_i} to a relative
  1e-8 the cut splits a cluster and m_i grows until it does not.
* Eigenvector sign: the entry of largest magnitude (lowest index on ties) is
  made positive.  M^{-1} does not depend on it.
* Krylov method: preconditioned CG (the paper uses GMRES with a 1e-6
  relative-residual stop).  Stop at the first k with
  ||r_k||_2 <= rtol ||f||_2 on the recurrence residual, x_0 = 0; iters = k.
  A flexible variant (Golub-Ye / Notay) uses
  beta_k = z_{k+1}^T (r_{k+1} - r_k) / (z_k^T r_k).
* Adjoint (not in the paper): lambda = A^{-1} g by the same PCG,
  dL/dA_ij = -lambda_i u_j on A's pattern, dL/df = lambda.
* Multiplicative two-grid cycle (the two-grid algorithm stated with the
  coarse space in Section 3.2: pre-smoothing, coarse-grid correction,
  post-smoothing; the Analysis of Section 4 carries its smoother constant
  C).  The paper names "a smoother S" without fixing it; this reading takes
  the local solves, damped: S = omega sum_i R_i^T A_i^{-1} R_i, the same
  smoother before and after the correction (so the cycle is symmetric),
  omega given by the caller (the cycle is SPD when
  0 < omega < 2 / lambda_max(sum_i R_i^T A_i^{-1} R_i A)).

Pins: every function here is checked against something other than itself
(closed forms, brute force on small inputs, library routines in the cases
the method reduces to them, the paper's lemmas and theorems, hand-worked
bfloat16 values) in tests/test_oracle_pins.py, and planted mistakes in
tests/test_oracle_mutations.py must fail those pins; no function is parity
unpinned.
"""

from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, List, Optional

import numpy as np
import scipy.linalg as la
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def csr_to_scipy(rowptr, colind, vals, n=None) -> sp.csr_matrix:
    n = len(rowptr) - 1 if n is None else n
    return sp.csr_matrix((np.asarray(vals, dtype=np.float64),
                          np.asarray(colind, dtype=np.int64),
                          np.asarray(rowptr, dtype=np.int64)), shape=(n, n))


# --------------------------------------------------------------------------
# Section 3.1: subdomains and Boolean restrictions R_i
# --------------------------------------------------------------------------

def index_maps(part: np.ndarray, nparts: int):
    """Dofs of each subdomain Omega_i (non-overlapping, Section 3.1).

    R_i picks the dofs with part == i in ascending global index.  Laid end
    to end over i = 0..N-1 they give ``perm`` (new position -> global dof);
    ``iperm`` is its inverse and ``sub_ptr[i]:sub_ptr[i+1]`` the range of
    subdomain i in that order.
    """
    part = np.asarray(part)
    n = part.shape[0]
    groups = [[] for _ in range(nparts)]
    for g in range(n):                 # ascending global index within each i
        groups[int(part[g])].append(g)
    perm = np.array([g for grp in groups for g in grp], dtype=np.int64)
    sub_ptr = np.zeros(nparts + 1, dtype=np.int64)
    sub_ptr[1:] = np.cumsum([len(grp) for grp in groups])
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n, dtype=np.int64)
    return perm, iperm, sub_ptr


# --------------------------------------------------------------------------
# Section 3.2: local matrices
# --------------------------------------------------------------------------

def local_matrices(A: sp.csr_matrix, dofs: np.ndarray):
    """A_i = R_i A R_i^T, \\hat A_i and the diagonal of S_i (Section 3.2).

    \\hat A_i keeps the off-diagonal entries of A_i and sets each diagonal
    entry to minus the sum of the off-diagonal entries of its row, so its
    row sums vanish.  S_i = diag(\\hat A_i); a zero S_jj is replaced by
    (A_i)_jj.
    """
    Ai = A[dofs][:, dofs].toarray()
    Ahat = Ai.copy()
    np.fill_diagonal(Ahat, 0.0)
    offsum = Ahat.sum(axis=1)
    np.fill_diagonal(Ahat, -offsum)
    s = np.diag(Ahat).copy()
    zero = s == 0.0
    s[zero] = np.diag(Ai)[zero]
    return Ai, Ahat, s


def local_eigenpairs(Ahat: np.ndarray, s: np.ndarray, m: int,
                     tie_rtol: float = 1e-8, all_pairs: bool = False,
                     threshold: Optional[float] = None):
    """Smallest eigenpairs of \\hat A_i psi = lambda S_i psi
    (Eq. algebraic-eigenproblem).

    Dense LAPACK generalized symmetric solver; eigenvectors come out
    S_i-orthonormal.  Returns ``(lam_all, Psi, m_i)`` with Psi of shape
    (n_i, m_i).  ``lam_all`` holds every computed eigenvalue (ascending).
    With ``threshold`` the count is adaptive: the modes with eigenvalue
    below it, at least one and at most m, so that lambda_{m_i+1} >= threshold
    wherever the cap does not bind (mu_c of Section 4 is then at least the
    threshold).
    """
    n_i = Ahat.shape[0]
    lam, V = la.eigh(Ahat, np.diag(s))
    m_i = min(m, n_i)
    if threshold is not None and m_i > 0:
        m_i = max(1, int(np.count_nonzero(lam[:m_i] < threshold)))
    while 0 < m_i < n_i and abs(lam[m_i] - lam[m_i - 1]) <= tie_rtol * max(abs(lam[m_i]), 1e-300):
        m_i += 1
    Psi = V[:, :m_i].copy()
    for k in range(m_i):
        j = int(np.argmax(np.abs(Psi[:, k])))        # lowest index on ties
        if Psi[j, k] < 0:
            Psi[:, k] = -Psi[:, k]
    return lam, Psi, m_i


def local_eigenpairs_hep(Ahat: np.ndarray, s: np.ndarray, m: int):
    """The same eigenpairs through the standard problem of Section 5.3:
    S^{-1/2} \\hat A S^{-1/2} z = lambda z, psi = S^{-1/2} z."""
    d = 1.0 / np.sqrt(s)
    H = Ahat * d[:, None] * d[None, :]
    lam, Z = la.eigh(H)
    return lam, Z[:, :m] * d[:, None]


# --------------------------------------------------------------------------
# Section 3.1-3.2: coarse space and Galerkin operator
# --------------------------------------------------------------------------

def coarse_basis(n: int, sub_dofs: List[np.ndarray], Psis: List[np.ndarray]) -> sp.csr_matrix:
    """R_0^T = [psi_1^(1) .. psi_{m_1}^(1), psi_1^(2) ..] with each local
    vector extended by zero outside its subdomain (Section 3.2)."""
    rows, cols, vals = [], [], []
    c0 = 0
    for dofs, Psi in zip(sub_dofs, Psis):
        ni, mi = Psi.shape
        for k in range(mi):
            rows.append(dofs)
            cols.append(np.full(ni, c0 + k, dtype=np.int64))
            vals.append(Psi[:, k])
        c0 += mi
    if c0 == 0:
        return sp.csr_matrix((n, 0))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, c0))


def coarse_matrix(A: sp.csr_matrix, R0T: sp.csr_matrix) -> np.ndarray:
    """Galerkin coarse matrix A_0 = R_0 A R_0^T (Section 3.1), dense."""
    return np.asarray((R0T.T @ (A @ R0T)).todense())


def round_basis(Psi: np.ndarray, mode: Optional[str]) -> np.ndarray:
    """Basis entries rounded to a storage precision (round to nearest, ties
    to even), directly from FP64.  Reading for the reduced-precision
    preconditioner: the coarse matrix is formed in FP64 from the rounded
    basis, so the coarse correction stays the exact Galerkin projection onto
    the stored space.

    bfloat16 keeps 8 significant bits and the exponent range of binary32:
    near |x| in [2^e-1, 2^e) its values are spaced 2^(e-8); below 2^-126
    (subnormal) the spacing stays 2^-133; magnitudes that round to 2^128 or
    beyond become infinite."""
    if mode is None:
        return Psi
    if mode == "fp32":
        return Psi.astype(np.float32).astype(np.float64)
    if mode == "bf16":
        Psi = np.asarray(Psi, dtype=np.float64)
        _, e = np.frexp(Psi)                  # Psi = m * 2^e, 0.5 <= |m| < 1
        q = np.maximum(e, -125) - 8           # spacing 2^q of the bfloat16 values there
        out = np.ldexp(np.rint(np.ldexp(Psi, -q)), q)
        return np.where(np.abs(out) >= 2.0 ** 128, np.copysign(np.inf, Psi), out)
    raise ValueError(mode)


# --------------------------------------------------------------------------
# the preconditioner and the Krylov solve
# --------------------------------------------------------------------------

@dataclass
class OracleAMS:
    """Setup of the two-level preconditioner on one SPD matrix.

    ``A`` scipy CSR; ``part`` subdomain id per dof; ``m`` eigenvectors per
    subdomain.  ``coarse=False`` drops the coarse term (block Jacobi)."""
    A: sp.csr_matrix
    part: np.ndarray
    nparts: int
    m: int
    coarse: bool = True
    tie_rtol: float = 1e-8
    basis_round: Optional[str] = None     # None, "fp32" or "bf16"
    eig_threshold: Optional[float] = None  # adaptive m_i (see local_eigenpairs)

    def __post_init__(self):
        A = self.A
        n = A.shape[0]
        self.n = n
        self.perm, self.iperm, self.sub_ptr = index_maps(self.part, self.nparts)
        self.sub_dofs = [self.perm[self.sub_ptr[i]:self.sub_ptr[i + 1]] for i in range(self.nparts)]
        self.local_chol = []
        self.lams, self.Psis, self.m_i = [], [], []
        for dofs in self.sub_dofs:
            Ai, Ahat, s = local_matrices(A, dofs)
            self.local_chol.append(la.cho_factor(Ai, lower=True))
            if self.coarse and self.m > 0:
                lam, Psi, mi = local_eigenpairs(Ahat, s, self.m, self.tie_rtol,
                                                threshold=self.eig_threshold)
            else:
                lam, Psi, mi = np.zeros(0), np.zeros((len(dofs), 0)), 0
            self.lams.append(lam)
            self.Psis.append(round_basis(Psi, self.basis_round))
            self.m_i.append(mi)
        self.R0T = coarse_basis(n, self.sub_dofs, self.Psis)
        self.Nc = self.R0T.shape[1]
        if self.Nc > 0:
            self.A0 = coarse_matrix(A, self.R0T)
            try:
                self.A0_chol = la.cho_factor(self.A0, lower=True)
            except la.LinAlgError as e:          # non-positive pivot
                raise ValueError("coarse matrix A_0 is not SPD") from e
        else:
            self.A0 = np.zeros((0, 0))
            self.A0_chol = None

    # M^{-1} r = sum_i R_i^T A_i^{-1} R_i r + R_0^T A_0^{-1} R_0 r
    def local_part(self, r: np.ndarray) -> np.ndarray:
        z = np.zeros_like(r)
        for dofs, ch in zip(self.sub_dofs, self.local_chol):
            z[dofs] = la.cho_solve(ch, r[dofs])
        return z

    def coarse_part(self, r: np.ndarray) -> np.ndarray:
        if self.Nc == 0:
            return np.zeros_like(r)
        rc = self.R0T.T @ r
        ec = la.cho_solve(self.A0_chol, rc)
        return self.R0T @ ec

    def apply(self, r: np.ndarray) -> np.ndarray:
        return self.local_part(r) + self.coarse_part(r)

    # One two-grid cycle for A x = r from x^0 = 0 (Section 3.2's two-grid
    # algorithm): x^1 = S r; coarse residual R_0 (r - A x^1), solved with
    # A_0 and added back through R_0^T; x^3 = x^2 + S (r - A x^2); with the
    # damped local solves as S.
    def apply_two_grid(self, r: np.ndarray, omega: float) -> np.ndarray:
        x1 = omega * self.local_part(r)
        x2 = x1 + self.coarse_part(r - self.A @ x1)
        return x2 + omega * self.local_part(r - self.A @ x2)

    def local_lambda_max(self) -> float:
        """Largest eigenvalue of T = (sum_i R_i^T A_i^{-1} R_i) A.  The sum of
        local solves is the inverse of the block-diagonal part D of A (its
        entries inside subdomains), so lambda_max(T) is the largest
        eigenvalue of the SPD pencil A x = lambda D x (Lanczos)."""
        A = self.A.tocoo()
        same = self.part[A.row] == self.part[A.col]
        D = sp.csr_matrix((A.data[same], (A.row[same], A.col[same])), shape=A.shape)
        Dinv = spla.LinearOperator(A.shape, matvec=self.local_part, dtype=np.float64)
        lam = spla.eigsh(self.A, k=1, M=D, Minv=Dinv, which="LA", tol=1e-12,
                         return_eigenvectors=False)
        return float(lam[0])

    def dense_Minv(self) -> np.ndarray:
        return np.column_stack([self.apply(e) for e in np.eye(self.n)])


@dataclass
class PCGResult:
    u: np.ndarray
    iters: int
    relres: float          # recurrence residual / ||f||
    true_relres: float     # ||f - A u|| / ||f||
    alphas: list
    betas: list
    converged: bool


def pcg(A: sp.csr_matrix, f: np.ndarray, Minv: Callable[[np.ndarray], np.ndarray],
        rtol: float = 1e-8, maxit: int = 10000, flexible: bool = False,
        x0: Optional[np.ndarray] = None) -> PCGResult:
    """Preconditioned CG from x_0 = 0, or from the initial guess x0
    (r_0 = f - A x_0), with the standard recurrences; flexible=True uses
    beta_k = z_{k+1}^T (r_{k+1} - r_k) / (z_k^T r_k).  The stop is relative
    to ||f|| whatever x_0 is; f = 0 gives x = 0."""
    f = np.asarray(f, dtype=np.float64)
    nf = np.linalg.norm(f)
    alphas, betas = [], []
    if nf == 0.0:
        return PCGResult(np.zeros_like(f), 0, 0.0, 0.0, alphas, betas, True)
    if x0 is None:
        x = np.zeros_like(f)
        r = f.copy()
    else:
        x = np.array(x0, dtype=np.float64, copy=True)
        r = f - A @ x
    z = Minv(r)
    p = z.copy()
    rz = r @ z
    k = 0
    converged = np.linalg.norm(r) <= rtol * nf
    while not converged and k < maxit:
        q = A @ p
        pq = p @ q
        alpha = rz / pq
        x = x + alpha * p
        r_old = r
        r = r - alpha * q
        k += 1
        alphas.append(alpha)
        if np.linalg.norm(r) <= rtol * nf:
            converged = True
            break
        z = Minv(r)
        if flexible:
            beta = (z @ (r - r_old)) / rz
        else:
            beta = (r @ z) / rz
        betas.append(beta)
        rz = r @ z
        p = z + beta * p
    true_res = np.linalg.norm(f - A @ x) / nf
    return PCGResult(x, k, float(np.linalg.norm(r) / nf), float(true_res),
                     alphas, betas, bool(converged))


def adjoint_gradient(A: sp.csr_matrix, u: np.ndarray, g: np.ndarray,
                     Minv: Callable, rtol: float = 1e-8, maxit: int = 10000):
    """Adjoint of u = A^{-1} f for a loss L(u) with dL/du = g.

    lambda = A^{-1} g (A symmetric, so A^T = A and the same preconditioner
    serves); dL/dA_ij = -lambda_i u_j on A's sparsity pattern, in CSR entry
    order; dL/df = lambda."""
    res = pcg(A, g, Minv, rtol=rtol, maxit=maxit)
    lam = res.u
    A = A.tocsr()
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    dvals = -lam[rows] * u[A.indices]
    return lam, dvals, res
