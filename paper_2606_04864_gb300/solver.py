"""Python binding of the AMS solve library (argument marshalling only).

Every computation runs in the CUDA library behind the C ABI of
``include/ams.h``; these classes only convert arrays, pass pointers and turn
status codes into exceptions.

Two pointer modes, fixed when a solver is built:

* host mode (``device=False``): NumPy arrays in and out; the library copies
  through its own device buffers.
* device mode (``device=True``): CUDA ``torch.Tensor`` in and out, passed to
  the library as device pointers on torch's current stream.

Vectors with several right-hand sides have shape ``(nrhs, n)`` (right-hand
side k is row k), which is the C ABI's n x nrhs column-major layout.
"""

from __future__ import annotations

import ctypes as C
from typing import List, Optional, Sequence

import numpy as np

from . import _lib
from ._lib import AMS_NUM_KERNELS, KERNEL_NAMES, AmsError, ams_info, ams_options, ams_system_desc, check, lib


def _torch():
    import torch
    return torch


def _stream_ptr(device: bool):
    if not device:
        return None
    torch = _torch()
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _as_host(a, dtype):
    try:
        torch = _torch()
        if isinstance(a, torch.Tensor):
            a = a.detach().cpu().numpy()
    except ImportError:  # pragma: no cover
        pass
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def _as_dev(a, dtype_np):
    torch = _torch()
    tdt = {np.float64: torch.float64, np.int64: torch.int64, np.int32: torch.int32}[dtype_np]
    if isinstance(a, torch.Tensor):
        return a.detach().to(device="cuda", dtype=tdt).contiguous()
    return torch.as_tensor(np.ascontiguousarray(a, dtype=dtype_np), device="cuda")


def _ptr(a):
    if isinstance(a, np.ndarray):
        return C.c_void_p(a.ctypes.data)
    return C.c_void_p(a.data_ptr())


def make_options(precision="fp32_bf16", cg="auto", maxit=10000, device=False, coarse=True,
                 eig_shift=0.0, eig_maxit=0, eig_tol=0.0, autotune=True, eig_threshold=0.0,
                 two_grid_omega=0.0, spin_budget_cycles=0, timeout_probe=False, warm_start=False) -> ams_options:
    o = ams_options()
    lib().ams_options_default(C.byref(o))
    o.precision = _lib.PREC[precision] if isinstance(precision, str) else int(precision)
    o.cg_variant = _lib.CG[cg] if isinstance(cg, str) else int(cg)
    o.maxit = int(maxit)
    o.device_ptrs = 1 if device else 0
    o.coarse = 1 if coarse else 0
    o.eig_shift = float(eig_shift)
    o.eig_maxit = int(eig_maxit)
    o.eig_tol = float(eig_tol)
    o.autotune = 1 if autotune else 0
    o.eig_threshold = float(eig_threshold)
    o.two_grid_omega = float(two_grid_omega)
    o.spin_budget_cycles = int(spin_budget_cycles)
    o.timeout_probe = 1 if timeout_probe else 0
    o.warm_start = 1 if warm_start else 0
    return o


class _Base:
    _h: Optional[C.c_void_p] = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def close(self):
        if self._h is not None and self._h.value:
            lib().ams_destroy(self._h)
        self._h = None

    def info(self) -> dict:
        i = ams_info()
        check(lib().ams_get_info(self._h, C.byref(i)), "ams_get_info")
        return {f: getattr(i, f) for f, _ in ams_info._fields_}

    _SHAPE_KEYS = ("bps_elem", "bps_sub", "depth", "nr", "l2mode", "l2keep")

    def launch_shape(self, nrhs: int = 1) -> dict:
        """Launch shapes used for solves with `nrhs` right-hand sides: blocks
        per SM of the element and subdomain grids, local-solve ring depth
        (0 = derived from the band width), right-hand sides per warp of the
        several-RHS local solve (0 = default), L2 priorities of the one-RHS
        local solve's tile copies (mode 0/1/2 and kept block rows), and
        whether they are fixed."""
        a = np.zeros(7, dtype=np.int32)
        check(lib().ams_get_launch_shape(self._h, int(nrhs), _ptr(a)), "ams_get_launch_shape")
        d = dict(zip(self._SHAPE_KEYS, (int(v) for v in a[:6])))
        d["fixed"] = bool(a[6])
        return d

    def set_launch_shape(self, nrhs: int = 1, **shape):
        """Fix the launch shapes for `nrhs` right-hand sides (keys as returned
        by launch_shape; missing keys keep their current value)."""
        cur = self.launch_shape(nrhs)
        a = np.array([int(shape.get(k, cur[k])) for k in self._SHAPE_KEYS], dtype=np.int32)
        check(lib().ams_set_launch_shape(self._h, int(nrhs), _ptr(a)), "ams_set_launch_shape")

    def _vec_in(self, v, nrhs_expected=None):
        if self.device:
            t = _as_dev(v, np.float64)
            if t.dim() == 1:
                t = t.unsqueeze(0)
            return t, t.shape[0]
        a = _as_host(v, np.float64)
        if a.ndim == 1:
            a = a[None, :]
        return np.ascontiguousarray(a), a.shape[0]

    def _check_out(self, out, nrhs):
        ok_shape = tuple(out.shape) in ((nrhs, self.n),) + (((self.n,),) if nrhs == 1 else ())
        if self.device:
            torch = _torch()
            ok = (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float64
                  and out.is_contiguous() and ok_shape)
        else:
            ok = (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags["C_CONTIGUOUS"]
                  and ok_shape)
        if not ok:
            raise ValueError(f"out must be a C-contiguous float64 ({nrhs}, {self.n}) "
                             f"{'CUDA tensor' if self.device else 'NumPy array'}")
        return out

    def _vec_out(self, nrhs):
        if self.device:
            return _torch().empty((nrhs, self.n), dtype=_torch().float64, device="cuda")
        return np.empty((nrhs, self.n), dtype=np.float64)

    def solve(self, f, rtol: float = 1e-8, allow_not_converged: bool = False, out=None, u0=None):
        """u = A^{-1} f by AMS-preconditioned CG.  Returns (u, iters, relres)
        with u shaped like f; iters/relres are int32/float64 arrays with one
        entry per (system,) right-hand side.  ``out``: optional (nrhs, n)
        float64 C-contiguous buffer of the solver's pointer mode to write u
        into (e.g. pinned host memory, so the copy back runs at full link
        speed).  ``u0``: initial guess, shaped like f (solvers built with
        warm_start=True; required there)."""
        fv, nrhs = self._vec_in(f)
        u = self._vec_out(nrhs) if out is None else self._check_out(out, nrhs)
        if self.opts.warm_start:
            if u0 is None:
                raise ValueError("this solver was built with warm_start=True: pass u0")
            u0v, n0 = self._vec_in(u0)
            if n0 != nrhs:
                raise ValueError("u0 needs as many right-hand sides as f")
            u.reshape(nrhs, self.n)[...] = u0v
        elif u0 is not None:
            raise ValueError("u0 needs a solver built with warm_start=True")
        its = np.zeros(self.nsys * nrhs, dtype=np.int32)
        rel = np.zeros(self.nsys * nrhs, dtype=np.float64)
        st = lib().ams_solve(self._h, _ptr(fv), nrhs, float(rtol), _ptr(u), _ptr(its), _ptr(rel))
        check(st, "ams_solve", allow=(4,) if allow_not_converged else ())
        if (hasattr(f, "ndim") and f.ndim == 1):
            u = u[0]
        return u, its, rel

    def profile_solve(self, f, rtol: float = 1e-8):
        """One solve with CUDA events around every kernel.  Returns one dict
        per kernel slot of the iteration (``KERNEL_NAMES`` order: SpMV with
        the direction update; local solves; coarse forward substitution,
        plus the backward one above four right-hand sides; prolongation with
        the CG update, plus the backward substitution up to four right-hand
        sides) with total ms, launch count and algorithmic bytes per launch."""
        fv, nrhs = self._vec_in(f)
        ms = np.zeros(AMS_NUM_KERNELS, dtype=np.float64)
        by = np.zeros(AMS_NUM_KERNELS, dtype=np.float64)
        cnt = np.zeros(AMS_NUM_KERNELS, dtype=np.int64)
        check(lib().ams_profile_solve(self._h, _ptr(fv), nrhs, float(rtol), _ptr(ms), _ptr(by), _ptr(cnt)),
              "ams_profile_solve", allow=(4,))
        return [{"name": KERNEL_NAMES[k], "ms": float(ms[k]), "count": int(cnt[k]), "bytes": float(by[k])}
                for k in range(AMS_NUM_KERNELS)]

    def time_kernel(self, which: int, reps: int = 20):
        ms = C.c_double()
        by = C.c_double()
        check(lib().ams_time_kernel(self._h, int(which), int(reps), C.byref(ms), C.byref(by)),
              "ams_time_kernel")
        return ms.value, by.value


def partition(rowptr, colind, nparts: int, imbalance: float = 0.0, seed: int = 0):
    """Built-in partition of a CSR pattern into `nparts` subdomains
    (``ams_partition``: multilevel recursive bisection, host code).  Returns
    (part int32[n], edge_cut)."""
    rp = np.ascontiguousarray(np.asarray(rowptr), dtype=np.int64)
    ci = np.ascontiguousarray(np.asarray(colind), dtype=np.int32)
    n = int(rp.shape[0] - 1)
    part = np.empty(max(n, 0), dtype=np.int32)
    cut = C.c_int64(0)
    check(lib().ams_partition(n, _ptr(rp), _ptr(ci), int(nparts), float(imbalance), int(seed), _ptr(part),
                              C.byref(cut)), "ams_partition")
    return part, int(cut.value)


class AmsSolver(_Base):
    """Two-level AMS preconditioner + CG on one sparse SPD matrix.

    Parameters follow ``ams_setup``: CSR arrays (rowptr int64, colind int32,
    vals float64), ``part`` (int32 subdomain id per dof, or None for the
    built-in partition of the pattern), ``nparts`` and ``m`` eigenvectors
    per subdomain.
    """

    def __init__(self, rowptr, colind, vals, part, nparts: int, m: int, precision="fp32_bf16",
                 cg="auto", maxit=10000, device: bool = False, coarse=True, eig_shift=0.0,
                 eig_maxit=0, eig_tol=0.0, autotune=True, eig_threshold=0.0, two_grid_omega=0.0,
                 spin_budget_cycles=0, timeout_probe=False, warm_start=False):
        self.device = bool(device)
        conv = _as_dev if self.device else _as_host
        self._rowptr = conv(rowptr, np.int64)
        self._colind = conv(colind, np.int32)
        self._vals = conv(vals, np.float64)
        self._part = conv(part, np.int32) if part is not None else None
        self.n = int(self._rowptr.shape[0] - 1)
        self.nnz = int(self._colind.shape[0])
        self.nparts = int(nparts)
        self.nsys = 1
        self.opts = make_options(precision, cg, maxit, self.device, coarse, eig_shift, eig_maxit, eig_tol,
                                 autotune, eig_threshold, two_grid_omega, spin_budget_cycles, timeout_probe,
                                 warm_start)
        h = C.c_void_p()
        st = lib().ams_setup(self.n, _ptr(self._rowptr), _ptr(self._colind), _ptr(self._vals),
                             _ptr(self._part) if self._part is not None else None, self.nparts, int(m),
                             C.byref(self.opts),
                             _stream_ptr(self.device), C.byref(h))
        check(st, "ams_setup")
        self._h = h
        # the library copied what it needs
        del self._rowptr, self._colind, self._vals, self._part

    def solve_adjoint(self, g, u, rtol: float = 1e-8, want_dvals: bool = True):
        """lambda = A^{-1} g and dL/dA_vals = -sum_k lambda_k[row] u_k[col]
        (CSR entry order).  Returns (lambda, dvals or None, iters)."""
        gv, nrhs = self._vec_in(g)
        uv, nu = self._vec_in(u)
        if nu != nrhs:
            raise ValueError("g and u need the same number of right-hand sides")
        lam = self._vec_out(nrhs)
        if want_dvals:
            dv = (_torch().empty(self.nnz, dtype=_torch().float64, device="cuda") if self.device
                  else np.empty(self.nnz, dtype=np.float64))
        else:
            dv = None
        its = np.zeros(nrhs, dtype=np.int32)
        st = lib().ams_solve_adjoint(self._h, _ptr(gv), nrhs, float(rtol), _ptr(uv), _ptr(lam),
                                     _ptr(dv) if dv is not None else None, _ptr(its))
        check(st, "ams_solve_adjoint")
        if hasattr(g, "ndim") and g.ndim == 1:
            lam = lam[0]
        return lam, dv, its

    def set_matrix_values(self, vals):
        """Replace A's values (same pattern) for later solves; the
        preconditioner built at setup is kept."""
        v = _as_dev(vals, np.float64) if self.device else _as_host(vals, np.float64)
        check(lib().ams_set_matrix_values(self._h, _ptr(v)), "ams_set_matrix_values")

    def index_maps(self):
        perm = np.empty(self.n, dtype=np.int64)
        sub_ptr = np.empty(self.nparts + 1, dtype=np.int64)
        check(lib().ams_get_index_maps(self._h, _ptr(perm), _ptr(sub_ptr)), "ams_get_index_maps")
        return perm, sub_ptr

    def coarse_basis(self):
        """(m_i, eigenvalues per subdomain, FP64 basis blocks per subdomain)."""
        mi = np.empty(self.nparts, dtype=np.int32)
        check(lib().ams_get_coarse_basis(self._h, _ptr(mi), None, None), "ams_get_coarse_basis")
        perm, sub_ptr = self.index_maps()
        ni = np.diff(sub_ptr)
        lam = np.empty(int(mi.sum()), dtype=np.float64)
        psi = np.empty(int((ni * mi).sum()), dtype=np.float64)
        check(lib().ams_get_coarse_basis(self._h, None, _ptr(lam), _ptr(psi)), "ams_get_coarse_basis")
        lams, psis = [], []
        lo = po = 0
        for i in range(self.nparts):
            lams.append(lam[lo:lo + mi[i]])
            blk = psi[po:po + ni[i] * mi[i]].reshape(mi[i], ni[i]).T.copy()
            psis.append(blk)
            lo += mi[i]
            po += ni[i] * mi[i]
        return mi, lams, psis

    def coarse_matrix(self):
        nc = int(self.info()["ncoarse"])
        A0 = np.empty((nc, nc), dtype=np.float64)
        check(lib().ams_get_coarse_matrix(self._h, _ptr(A0)), "ams_get_coarse_matrix")
        return A0

    def coarse_factor_inverse(self):
        """(L_c^{-1} in the coarse solve's nested-dissection order, nd_paper):
        ``nd_paper[p]`` is the paper-order coarse index of ND position p."""
        nc = int(self.info()["ncoarse"])
        Linv = np.empty((nc, nc), dtype=np.float64)
        order = np.empty(nc, dtype=np.int64)
        check(lib().ams_get_coarse_factor_inverse(self._h, _ptr(order), _ptr(Linv)),
              "ams_get_coarse_factor_inverse")
        return Linv, order

    def apply_preconditioner(self, r):
        rv, nrhs = self._vec_in(r)
        z = self._vec_out(nrhs)
        check(lib().ams_apply_preconditioner(self._h, _ptr(rv), nrhs, _ptr(z)), "ams_apply_preconditioner")
        return z[0] if (hasattr(r, "ndim") and r.ndim == 1) else z

    def spmv(self, x):
        xv, nrhs = self._vec_in(x)
        y = self._vec_out(nrhs)
        check(lib().ams_spmv(self._h, _ptr(xv), nrhs, _ptr(y)), "ams_spmv")
        return y[0] if (hasattr(x, "ndim") and x.ndim == 1) else y


class AmsBatchedSolver(_Base):
    """Several independent systems solved together (``ams_setup_batched``).

    ``systems`` is a sequence of (rowptr, colind, vals, part, nparts, m);
    ``part=None`` takes the built-in partition of that system's pattern.
    The C ABI lays the systems' n_s x nrhs column-major blocks end to end;
    :meth:`pack` and :meth:`unpack` convert from and to lists of per-system
    (nrhs, n_s) arrays.
    """

    def __init__(self, systems: Sequence, precision="fp32_bf16", cg="auto", maxit=10000,
                 device: bool = False, coarse=True, autotune=True, eig_threshold=0.0):
        self.device = bool(device)
        conv = _as_dev if self.device else _as_host
        keep = []
        descs = (ams_system_desc * len(systems))()
        self.sizes = []
        for k, (rowptr, colind, vals, part, nparts, m) in enumerate(systems):
            arrs = (conv(rowptr, np.int64), conv(colind, np.int32), conv(vals, np.float64),
                    conv(part, np.int32) if part is not None else None)
            keep.append(arrs)
            n = int(arrs[0].shape[0] - 1)
            self.sizes.append(n)
            descs[k] = ams_system_desc(n, _ptr(arrs[0]), _ptr(arrs[1]), _ptr(arrs[2]),
                                       _ptr(arrs[3]) if arrs[3] is not None else None, int(nparts), int(m))
        self.n = int(sum(self.sizes))
        self.nsys = len(systems)
        self.opts = make_options(precision, cg, maxit, self.device, coarse, autotune=autotune,
                                 eig_threshold=eig_threshold)
        h = C.c_void_p()
        st = lib().ams_setup_batched(self.nsys, descs, C.byref(self.opts), _stream_ptr(self.device),
                                     C.byref(h))
        check(st, "ams_setup_batched")
        self._h = h

    def pack(self, blocks: List):
        """List of per-system (nrhs, n_s) arrays -> flat buffer of the ABI layout."""
        if self.device:
            torch = _torch()
            return torch.cat([_as_dev(b, np.float64).reshape(-1) for b in blocks])
        return np.concatenate([np.ascontiguousarray(b, dtype=np.float64).reshape(-1) for b in blocks])

    def unpack(self, flat, nrhs: int):
        out, o = [], 0
        for n in self.sizes:
            out.append(flat[o:o + n * nrhs].reshape(nrhs, n))
            o += n * nrhs
        return out

    def profile_solve(self, f_flat, nrhs: int, rtol: float = 1e-8):
        """As :meth:`AmsSolver.profile_solve`, for f_flat in the ABI layout."""
        fv = _as_dev(f_flat, np.float64) if self.device else _as_host(f_flat, np.float64)
        ms = np.zeros(AMS_NUM_KERNELS, dtype=np.float64)
        by = np.zeros(AMS_NUM_KERNELS, dtype=np.float64)
        cnt = np.zeros(AMS_NUM_KERNELS, dtype=np.int64)
        check(lib().ams_profile_solve(self._h, _ptr(fv), int(nrhs), float(rtol), _ptr(ms), _ptr(by), _ptr(cnt)),
              "ams_profile_solve", allow=(4,))
        return [{"name": KERNEL_NAMES[k], "ms": float(ms[k]), "count": int(cnt[k]), "bytes": float(by[k])}
                for k in range(AMS_NUM_KERNELS)]

    def solve(self, f_flat, nrhs: int, rtol: float = 1e-8, allow_not_converged: bool = False, out=None):
        """f_flat in the ABI layout (see :meth:`pack`).  Returns (u_flat,
        iters[nsys, nrhs], relres[nsys, nrhs]).  ``out``: optional float64
        C-contiguous buffer shaped like f_flat, of the solver's pointer mode,
        to write u into (e.g. pinned host memory)."""
        fv = _as_dev(f_flat, np.float64) if self.device else _as_host(f_flat, np.float64)
        if out is None:
            u = (_torch().empty_like(fv) if self.device else np.empty_like(fv))
        else:
            torch = _torch() if self.device else None
            ok = (tuple(out.shape) == tuple(fv.shape) and
                  ((isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float64
                    and out.is_contiguous()) if self.device else
                   (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags["C_CONTIGUOUS"])))
            if not ok:
                raise ValueError("out must be a C-contiguous float64 buffer shaped like f_flat, "
                                 + ("a CUDA tensor" if self.device else "a host array"))
            u = out
        its = np.zeros(self.nsys * nrhs, dtype=np.int32)
        rel = np.zeros(self.nsys * nrhs, dtype=np.float64)
        st = lib().ams_solve(self._h, _ptr(fv), int(nrhs), float(rtol), _ptr(u), _ptr(its), _ptr(rel))
        check(st, "ams_solve", allow=(4,) if allow_not_converged else ())
        return u, its.reshape(self.nsys, nrhs), rel.reshape(self.nsys, nrhs)
