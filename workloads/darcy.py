"""TPFA Darcy matrices, permeability fields and partitions (seeded, synthetic).

Grid convention: a ``d``-dimensional grid of ``shape = (nz, ny, nx)`` (3-D) or
``(ny, nx)`` (2-D) cells on the unit square/cube, cell size ``h = 1/side``,
flat cell index ``(iz*ny + iy)*nx + ix`` (x fastest).  Arrays holding one value
per cell use that same C order.

Matrix: the two-point flux finite-volume discretisation of
``-div(kappa grad u) = f`` with homogeneous Dirichlet data.  An interior face
between cells i and j carries ``T = h^(d-2) * 2 k_i k_j / (k_i + k_j)`` (the
harmonic mean over a distance h through an area h^(d-1)); a boundary face of
cell i carries ``T_b = h^(d-2) * 2 k_i`` (half-cell distance to the Dirichlet
wall).  ``A_ij = -T`` for each interior face and ``A_ii`` is the sum of all face
transmissibilities of cell i, so A is a symmetric M-matrix with non-negative
row sums (strictly positive on boundary rows): the class of matrices the
paper's analysis assumes (Section 4, Lemma 2).  The right-hand side
``f_i = h^d`` integrates a unit source over the cell.

CSR layout: row i lists its entries in ascending column order, which on this
grid is (-z, -y, -x, diagonal, +x, +y, +z) with missing neighbours skipped;
``rowptr`` is int64, ``colind`` int32 and ``vals`` float64.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
from scipy import ndimage


# --------------------------------------------------------------------------
# permeability fields
# --------------------------------------------------------------------------

def grf_logk(shape, sigma: float, std: float, seed: int) -> np.ndarray:
    """Gaussian random field for log-permeability.

    Seeded N(0,1) white noise, smoothed by a Gaussian filter of ``sigma``
    cells (reflecting boundaries, kernel truncated at 4 sigma), shifted to
    zero mean and rescaled to the exact target standard deviation.
    """
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(tuple(shape))
    sm = ndimage.gaussian_filter(noise, sigma=sigma, mode="reflect", truncate=4.0)
    sm = sm - sm.mean()
    s = sm.std()
    if s > 0:
        sm = sm * (std / s)
    return np.ascontiguousarray(sm, dtype=np.float64)


def channel_field(shape, nchannels: int = 200, kmax: float = 1e6,
                  wmin: int = 2, wmax: int = 4, lmin: int = 64, lmax: int = 512,
                  seed: int = 0) -> np.ndarray:
    """High-contrast channelised log-permeability on a 2-D grid.

    Background k = 1; ``nchannels`` axis-aligned rectangles (orientation x or
    y with probability 1/2, width uniform in [wmin, wmax], length uniform in
    [lmin, lmax], lower-left corner uniform over the grid, clipped at the
    domain) are set to ``kmax``.  Stands in for the paper's channel images
    (Section 5.1), which are not available.  Returns log k.
    """
    ny, nx = shape
    rng = np.random.default_rng(seed)
    k = np.ones((ny, nx), dtype=np.float64)
    for _ in range(nchannels):
        orient = int(rng.integers(0, 2))
        width = int(rng.integers(wmin, wmax + 1))
        length = int(rng.integers(lmin, lmax + 1))
        x0 = int(rng.integers(0, nx))
        y0 = int(rng.integers(0, ny))
        if orient == 0:
            k[y0:y0 + width, x0:x0 + length] = kmax
        else:
            k[y0:y0 + length, x0:x0 + width] = kmax
    return np.log(k)


# --------------------------------------------------------------------------
# TPFA assembly
# --------------------------------------------------------------------------

@dataclass
class FaceList:
    """Face-to-CSR map of a TPFA grid (used for assembly and for chaining
    matrix-value gradients back to the permeability)."""
    shape: tuple
    h: float
    hfac: float                 # h^(d-2)
    fi: np.ndarray              # interior faces: lower cell
    fj: np.ndarray              # interior faces: upper cell
    pos_ij: np.ndarray          # CSR position of (fi, fj)
    pos_ji: np.ndarray          # CSR position of (fj, fi)
    pos_ii: np.ndarray          # CSR position of (fi, fi)
    pos_jj: np.ndarray          # CSR position of (fj, fj)
    bcell: np.ndarray           # one entry per boundary face: its cell
    pos_b: np.ndarray           # CSR position of (bcell, bcell)
    rowptr: np.ndarray
    colind: np.ndarray


def tpfa_face_list(shape) -> FaceList:
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    assert d in (2, 3)
    n = int(np.prod(shape))
    side = max(shape)
    h = 1.0 / side
    hfac = h ** (d - 2)
    # axis a (0 = x fastest); stride and coordinate of each cell along a
    idx = np.arange(n, dtype=np.int64)
    coords = np.unravel_index(idx, shape)          # (.., iy, ix) in C order
    axes = []                                      # x, y, (z)
    stride = 1
    for a in range(d):
        c = coords[d - 1 - a]
        axes.append((stride, c, shape[d - 1 - a]))
        stride *= shape[d - 1 - a]
    # slots in ascending column order: -z,-y,-x, diag, +x,+y,+z
    slots = []
    for a in reversed(range(d)):
        st, c, L = axes[a]
        slots.append(("m", a, c > 0, -st))
    slots.append(("d", -1, np.ones(n, dtype=bool), 0))
    for a in range(d):
        st, c, L = axes[a]
        slots.append(("p", a, c < L - 1, st))
    masks = np.stack([s[2] for s in slots])        # (nslots, n)
    counts = masks.sum(axis=0).astype(np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    before = np.cumsum(masks, axis=0) - masks      # entries before slot s in row
    pos = rowptr[:-1][None, :] + before            # (nslots, n)
    nnz = int(rowptr[-1])
    colind = np.empty(nnz, dtype=np.int32)
    for s, (kind, a, m, off) in enumerate(slots):
        colind[pos[s][m]] = (idx[m] + off).astype(np.int32)
    dslot = d
    pos_diag = pos[dslot]
    fi_l, fj_l, pij_l, pji_l = [], [], [], []
    for a in range(d):
        st = axes[a][0]
        sp = dslot + 1 + a                        # +a slot of the lower cell
        sm = d - 1 - a                            # -a slot of the upper cell
        m = masks[sp]
        i = idx[m]
        j = i + st
        fi_l.append(i)
        fj_l.append(j)
        pij_l.append(pos[sp][m])
        pji_l.append(pos[sm][j])
    fi = np.concatenate(fi_l)
    fj = np.concatenate(fj_l)
    bc_l = []
    for a in range(d):
        st, c, L = axes[a]
        bc_l.append(idx[c == 0])
        bc_l.append(idx[c == L - 1])
    bcell = np.concatenate(bc_l)
    return FaceList(shape=shape, h=h, hfac=hfac, fi=fi, fj=fj,
                    pos_ij=np.concatenate(pij_l), pos_ji=np.concatenate(pji_l),
                    pos_ii=pos_diag[fi], pos_jj=pos_diag[fj],
                    bcell=bcell, pos_b=pos_diag[bcell],
                    rowptr=rowptr, colind=colind)


def tpfa_csr(logk: np.ndarray, faces: Optional[FaceList] = None):
    """Assemble the TPFA matrix for ``kappa = exp(logk)``.

    Returns ``(rowptr int64, colind int32, vals float64)``.  The matrix is
    exactly symmetric (both triangles receive the same rounded T).
    """
    if faces is None:
        faces = tpfa_face_list(logk.shape)
    k = np.exp(logk.reshape(-1))
    ki = k[faces.fi]
    kj = k[faces.fj]
    T = faces.hfac * 2.0 * ki * kj / (ki + kj)
    Tb = faces.hfac * 2.0 * k[faces.bcell]
    nnz = faces.colind.shape[0]
    vals = np.zeros(nnz, dtype=np.float64)
    vals[faces.pos_ij] = -T
    vals[faces.pos_ji] = -T
    np.add.at(vals, faces.pos_ii, T)
    np.add.at(vals, faces.pos_jj, T)
    np.add.at(vals, faces.pos_b, Tb)
    return faces.rowptr, faces.colind, vals


def tpfa_values_from_logk(logk, faces: FaceList):
    """Differentiable (torch) TPFA assembly: CSR values as a function of a
    torch tensor ``logk`` (flat, one value per cell).  Same formulas and
    CSR layout as :func:`tpfa_csr`; used to chain dL/dA_vals to dL/dlog k."""
    import torch
    dev = logk.device
    k = torch.exp(logk.reshape(-1))
    fi = torch.as_tensor(faces.fi, device=dev)
    fj = torch.as_tensor(faces.fj, device=dev)
    bc = torch.as_tensor(faces.bcell, device=dev)
    ki = k[fi]
    kj = k[fj]
    T = faces.hfac * 2.0 * ki * kj / (ki + kj)
    Tb = faces.hfac * 2.0 * k[bc]
    nnz = faces.colind.shape[0]
    vals = torch.zeros(nnz, dtype=logk.dtype, device=dev)
    vals = vals.index_add(0, torch.as_tensor(faces.pos_ij, device=dev), -T)
    vals = vals.index_add(0, torch.as_tensor(faces.pos_ji, device=dev), -T)
    vals = vals.index_add(0, torch.as_tensor(faces.pos_ii, device=dev), T)
    vals = vals.index_add(0, torch.as_tensor(faces.pos_jj, device=dev), T)
    vals = vals.index_add(0, torch.as_tensor(faces.pos_b, device=dev), Tb)
    return vals


# --------------------------------------------------------------------------
# partitions
# --------------------------------------------------------------------------

def block_partition(shape, bs: int):
    """Regular block partition: blocks of ``bs`` cells per axis (the last
    block along an axis is partial when bs does not divide the side).  Block
    ids run over the block grid in the same C order as cells.  Returns
    ``(part int32[n], nparts)``."""
    shape = tuple(int(s) for s in shape)
    nb = [(s + bs - 1) // bs for s in shape]
    grids = np.meshgrid(*[np.arange(s) // bs for s in shape], indexing="ij")
    part = np.zeros(shape, dtype=np.int64)
    for ax in range(len(shape)):
        part = part * nb[ax] + grids[ax]
    return part.reshape(-1).astype(np.int32), int(np.prod(nb))


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    shape: tuple
    logk: np.ndarray
    rowptr: np.ndarray
    colind: np.ndarray
    vals: np.ndarray
    part: np.ndarray
    nparts: int
    m: int
    rhs: np.ndarray            # (nrhs, n) C order: RHS k is rhs[k]
    rtol: float = 1e-8
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.rowptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.colind.shape[0])

    @property
    def nrhs(self) -> int:
        return int(self.rhs.shape[0])


def _build(name, logk, bs, m, rhs_kind, nrhs, seed, rtol=1e-8):
    shape = logk.shape
    faces = tpfa_face_list(shape)
    rowptr, colind, vals = tpfa_csr(logk, faces)
    part, nparts = block_partition(shape, bs)
    n = int(np.prod(shape))
    h = faces.h
    if rhs_kind == "unit":
        rhs = np.full((nrhs, n), h ** len(shape), dtype=np.float64)
    else:
        rng = np.random.default_rng(seed + 7919)
        rhs = rng.standard_normal((nrhs, n))
    return Workload(name=name, shape=tuple(shape), logk=logk, rowptr=rowptr,
                    colind=colind, vals=vals, part=part, nparts=nparts, m=m,
                    rhs=np.ascontiguousarray(rhs), rtol=rtol,
                    extra={"faces": faces, "bs": bs})


def make_from_logk(name, logk, bs, m, rhs_kind="unit", nrhs=1, seed=0):
    """Workload on a given log-permeability array (e.g. a window of a larger
    field, used for bounded CPU samples of a full-size workload)."""
    return _build(name, np.ascontiguousarray(logk), bs, m, rhs_kind, nrhs, seed)


def make_small_2d(side=16, bs=4, m=2, std=1.0, sigma=2.0, seed=0, nrhs=1,
                  rhs_kind="unit", ny=None):
    shape = (ny if ny is not None else side, side)
    logk = grf_logk(shape, sigma, std, seed)
    return _build(f"small2d_{shape[0]}x{shape[1]}_b{bs}_m{m}", logk, bs, m,
                  rhs_kind, nrhs, seed)


def make_small_3d(side=8, bs=4, m=2, std=1.0, sigma=2.0, seed=0, nrhs=1,
                  rhs_kind="unit"):
    shape = (side, side, side)
    logk = grf_logk(shape, sigma, std, seed)
    return _build(f"small3d_{side}_b{bs}_m{m}", logk, bs, m, rhs_kind, nrhs,
                  seed)


def make_grf2d_64():
    """2-D 64x64 GRF Darcy (sigma 4, log-std 2), 8x8 blocks, m=4, 1 RHS."""
    logk = grf_logk((64, 64), sigma=4.0, std=2.0, seed=1)
    return _build("darcy2d_64x64_grf_b8_m4", logk, 8, 4, "unit", 1, 1)


def make_channels2d_1024(side=1024):
    """2-D 1024x1024 channelised Darcy (200 channels, k=1e6), 32x32 blocks,
    m=8, 1 RHS."""
    logk = channel_field((side, side), nchannels=200, kmax=1e6, seed=2)
    return _build(f"darcy2d_{side}x{side}_channels1e6_b32_m8", logk, 32, 8,
                  "unit", 1, 2)


def make_grf3d_128_rhs32(side=128, nrhs=32):
    """3-D 128^3 lognormal Darcy (log-std 3, sigma 6), 8^3 blocks, m=6,
    32 RHS iid N(0,1)."""
    logk = grf_logk((side, side, side), sigma=6.0, std=3.0, seed=3)
    return _build(f"darcy3d_{side}^3_grf_b8_m6_rhs{nrhs}", logk, 8, 6, "normal",
                  nrhs, 3)


def make_batch48_uneven(nsys2d=24, nsys3d=24, lo2=128, hi2=512, lo3=32, hi3=96,
                 nrhs=8, seed=4) -> List[Workload]:
    """48 uneven systems: 2-D sides U[128,512] and 3-D sides U[32,96],
    log-std U[2,3], 8^d blocks (partial at the far edges), m U{4..8},
    8 RHS iid N(0,1) each."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(nsys2d + nsys3d):
        is3 = s >= nsys2d
        side = int(rng.integers(lo3, hi3 + 1)) if is3 else int(rng.integers(lo2, hi2 + 1))
        std = float(rng.uniform(2.0, 3.0))
        m = int(rng.integers(4, 9))
        sub = int(rng.integers(0, 2**31 - 1))
        shape = (side,) * (3 if is3 else 2)
        logk = grf_logk(shape, 6.0 if is3 else 4.0, std, sub)
        out.append(_build(f"sys{s}_{'3d' if is3 else '2d'}_{side}", logk, 8, m,
                          "normal", nrhs, sub))
    return out


def make_grf3d_96_adjoint(side=96, nobs=4096, seed=5):
    """3-D 96^3 lognormal Darcy (log-std 2, sigma 6), f=1, 8^3 blocks, m=6.

    ``extra`` holds the observation cells (``obs``, drawn without
    replacement) and the perturbed truth field ``logk_truth = logk + xi``
    (xi an independent GRF, sigma 6, std 0.5); the data vector d is the
    truth field's solution at ``obs`` and is computed by whoever holds a
    solver."""
    logk = grf_logk((side,) * 3, sigma=6.0, std=2.0, seed=seed)
    w = _build(f"darcy3d_{side}^3_grf_b8_m6_adjoint", logk, 8, 6, "unit", 1,
               seed)
    xi = grf_logk((side,) * 3, sigma=6.0, std=0.5, seed=seed + 101)
    rng = np.random.default_rng(seed + 202)
    obs = np.sort(rng.choice(w.n, size=min(nobs, w.n), replace=False)).astype(np.int64)
    w.extra.update({"obs": obs, "logk_truth": logk + xi})
    return w
