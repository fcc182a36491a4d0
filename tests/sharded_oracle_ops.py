"""Per-rank operations of the sharded iteration built from the CPU oracle
(test infrastructure): the rank's rows of A from the plan, and the oracle's
local Cholesky factors, basis blocks and coarse factor for its subdomains.
Vectors are 1-D, or blocks with one column per right-hand side."""

import numpy as np
import scipy.linalg as la
import scipy.sparse as sp


class OracleRankOps:
    def __init__(self, o, plan, rank):
        rp = plan.ranks[rank]
        self.rp, self.o, self.plan = rp, o, plan
        self.A = sp.csr_matrix((rp.vals, rp.colind, rp.rowptr), shape=(rp.n_owned, rp.n_owned + len(rp.ghost)))
        self.subs = [(i, int(plan.sub_ptr[i] - rp.row_lo), int(plan.sub_ptr[i + 1] - rp.row_lo),
                      int(plan.coarse_ptr[i]), int(plan.coarse_ptr[i + 1])) for i in range(rp.sub_lo, rp.sub_hi)]

    def spmv(self, p_owned, p_ghost):
        return self.A @ np.concatenate([p_owned, p_ghost])

    def local_restrict(self, r):
        zf = np.zeros_like(r)
        rc = np.zeros((self.rp.coarse_hi - self.rp.coarse_lo,) + r.shape[1:])
        for i, a, b, c0, c1 in self.subs:
            zf[a:b] = la.cho_solve(self.o.local_chol[i], r[a:b])
            rc[c0 - self.rp.coarse_lo:c1 - self.rp.coarse_lo] = self.o.Psis[i].T @ r[a:b]
        return zf, rc

    def coarse_solve(self, rc_full):
        return la.cho_solve(self.o.A0_chol, rc_full)

    def prolong(self, zf, ec_full):
        z = zf.copy()
        for i, a, b, c0, c1 in self.subs:
            z[a:b] += self.o.Psis[i] @ ec_full[c0:c1]
        return z

    def sddmm(self, lam, u_owned, u_ghost):
        uext = np.concatenate([u_owned, u_ghost])
        rows = np.repeat(np.arange(self.rp.n_owned), np.diff(self.rp.rowptr))
        prod = lam[rows] * uext[self.rp.colind]
        return -(prod if prod.ndim == 1 else prod.sum(axis=1))

    def dot(self, a, b):
        return float(a @ b) if a.ndim == 1 else np.einsum("ij,ij->j", a, b)

    def axpy(self, alpha, x, y):
        return y + alpha * x

    def copy(self, x):
        return np.array(x, dtype=np.float64, copy=True)

    def zeros_like(self, x):
        return np.zeros_like(x)

    def gather(self, x, idx):
        return np.asarray(x)[idx]
