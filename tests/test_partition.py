"""The built-in partitioner (ams_partition): valid, balanced, deterministic
partitions with cuts close to the best possible on meshes, and the optimum
on small graphs where it is known.  Host code only: runs without a GPU.

The method takes the subdomain partition as an input (Section 3.1; the
paper's experiments use METIS); these tests hold the partitioner to what
any such partition must satisfy and to known optimal cuts, not to METIS."""

import math

import numpy as np
import pytest
import scipy.sparse as sp


@pytest.fixture(scope="module")
def partition():
    from paper_2606_04864_gb300._build import build
    build()
    from paper_2606_04864_gb300 import partition as p
    return p


def _csr(n, edges, diag=True, symmetric=True):
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    i, j = edges[:, 0], edges[:, 1]
    if symmetric:
        i, j = np.concatenate([i, j]), np.concatenate([j, i])
    A = sp.coo_matrix((np.ones(len(i)), (i, j)), shape=(n, n)).tocsr()
    if diag:
        A = (A + sp.eye(n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A.indptr.astype(np.int64), A.indices.astype(np.int32)


def _grid_edges(shape):
    idx = np.arange(int(np.prod(shape))).reshape(shape)
    out = []
    for ax in range(len(shape)):
        a = np.moveaxis(idx, ax, 0)
        out.append(np.stack([a[:-1].ravel(), a[1:].ravel()], axis=1))
    return np.concatenate(out)


def _cut(rowptr, colind, part):
    rows = np.repeat(np.arange(len(rowptr) - 1), np.diff(rowptr))
    off = rows != colind
    e = {(min(a, b), max(a, b)) for a, b in zip(rows[off], colind[off])}
    return sum(part[a] != part[b] for a, b in e)


def _check_valid(part, n, k, imbalance=0.03):
    assert part.shape == (n,) and part.dtype == np.int32
    assert part.min() >= 0 and part.max() < k
    sizes = np.bincount(part, minlength=k)
    assert sizes.min() >= 1
    bound = (1 + imbalance) * n / k + max(1, math.ceil(math.log2(max(k, 2))))
    assert sizes.max() <= bound, (sizes.max(), bound)
    return sizes


def test_grid_2d_cut_balance_and_reported_cut(partition):
    """64 x 64 grid into 16 parts: the 4 x 4 block partition cuts 384
    edges and no balanced 16-way partition does much better."""
    rp, ci = _csr(64 * 64, _grid_edges((64, 64)))
    part, cut = partition(rp, ci, 16)
    _check_valid(part, 64 * 64, 16)
    assert cut == _cut(rp, ci, part)
    assert cut <= 1.10 * 384


def test_grid_3d_cut(partition):
    """16^3 grid into 8 parts: the 2 x 2 x 2 block partition cuts
    3 * 16^2 = 768 edges."""
    rp, ci = _csr(16 ** 3, _grid_edges((16, 16, 16)))
    part, cut = partition(rp, ci, 8)
    _check_valid(part, 16 ** 3, 8)
    assert cut == _cut(rp, ci, part)
    assert cut <= 1.05 * 768


@pytest.mark.parametrize("n,k,edges,best", [
    (8, 2, [(i, i + 1) for i in range(7)], 1),                      # path: one cut edge
    (12, 3, [(i, (i + 1) % 12) for i in range(12)], 3),             # cycle: one edge per part boundary
    (16, 2, _grid_edges((4, 4)).tolist(), 4),                       # 4 x 4 grid: a straight line
    (10, 2, [(i, j) for i in range(5) for j in range(i + 1, 5)] +   # two 5-cliques and a bridge
     [(i, j) for i in range(5, 10) for j in range(i + 1, 10)] + [(4, 5)], 1),
])
def test_small_graphs_reach_the_optimum(partition, n, k, edges, best):
    rp, ci = _csr(n, edges)
    part, cut = partition(rp, ci, k, imbalance=0.0)
    sizes = _check_valid(part, n, k)
    assert sizes.max() - sizes.min() <= 1
    assert cut == best == _cut(rp, ci, part)


def test_degenerate_cases(partition):
    # one part, and one dof per part
    rp, ci = _csr(30, [(i, i + 1) for i in range(29)])
    part, cut = partition(rp, ci, 1)
    assert (part == 0).all() and cut == 0
    part, cut = partition(rp, ci, 30)
    assert sorted(part.tolist()) == list(range(30)) and cut == 29
    # no off-diagonal entries: any balanced assignment, nothing cut
    rp, ci = _csr(50, np.zeros((0, 2)))
    part, cut = partition(rp, ci, 7)
    _check_valid(part, 50, 7)
    assert cut == 0
    # two disconnected grids and isolated dofs, split into 5
    e = np.concatenate([_grid_edges((10, 10)), _grid_edges((8, 8)) + 100])
    rp, ci = _csr(100 + 64 + 6, e)
    part, cut = partition(rp, ci, 5)
    _check_valid(part, 170, 5)
    assert cut == _cut(rp, ci, part)


def test_deterministic_and_seeded(partition):
    rp, ci = _csr(40 * 40, _grid_edges((40, 40)))
    a, ca = partition(rp, ci, 12, seed=7)
    b, cb = partition(rp, ci, 12, seed=7)
    assert np.array_equal(a, b) and ca == cb
    c, cc = partition(rp, ci, 12, seed=8)
    _check_valid(c, 1600, 12)
    assert cc == _cut(rp, ci, c)


def test_one_triangle_of_the_pattern_gives_the_same_graph(partition):
    """The pattern is symmetrised: the upper triangle alone describes the
    same graph as the full symmetric pattern."""
    e = _grid_edges((20, 20))
    rp, ci = _csr(400, e)
    ru, cu = _csr(400, np.sort(e, axis=1), symmetric=False)
    a, ca = partition(rp, ci, 6)
    b, cb = partition(ru, cu, 6)
    assert np.array_equal(a, b) and ca == cb


def test_looser_imbalance_is_respected(partition):
    rp, ci = _csr(30 * 30, _grid_edges((30, 30)))
    part, _ = partition(rp, ci, 7, imbalance=0.10)
    _check_valid(part, 900, 7, imbalance=0.10)


def test_invalid_arguments_are_rejected(partition):
    from paper_2606_04864_gb300._lib import AmsError
    rp, ci = _csr(10, [(i, i + 1) for i in range(9)])
    for kw in ({"nparts": 0}, {"nparts": 11}, {"nparts": 2, "imbalance": -0.1},
               {"nparts": 2, "imbalance": float("nan")}):
        with pytest.raises(AmsError):
            partition(rp, ci, kw.pop("nparts"), **kw)
    bad = ci.copy()
    bad[3] = 10
    with pytest.raises(AmsError):
        partition(rp, bad, 2)
    rp2 = rp.copy()
    rp2[5] = rp2[6] + 1
    with pytest.raises(AmsError):
        partition(rp2, ci, 2)
