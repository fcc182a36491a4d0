"""The byte model behind the bench's roofline: nested-dissection factor
counts checked against the structure of actual dense Cholesky factors."""

import numpy as np
import pytest

import bench


def _grid_matrix(shape, rng, weights=None):
    """Random SPD matrix with the (2d+1)-point grid pattern; with weights,
    each cell is a dense block of that many unknowns coupled densely to the
    blocks of its face neighbours."""
    n = int(np.prod(shape))
    wt = np.ones(n, dtype=int) if weights is None else np.asarray(weights)
    off = np.concatenate([[0], np.cumsum(wt)])
    N = int(off[-1])
    M = np.zeros((N, N))
    idx = np.arange(n).reshape(shape)
    for ax in range(len(shape)):
        a = np.moveaxis(idx, ax, 0)
        for i, j in zip(a[:-1].ravel(), a[1:].ravel()):
            blk = -rng.uniform(0.5, 1.5, (wt[i], wt[j]))
            M[off[i]:off[i + 1], off[j]:off[j + 1]] = blk
            M[off[j]:off[j + 1], off[i]:off[i + 1]] = blk.T
    for i in range(n):
        B = rng.uniform(-0.1, 0.1, (wt[i], wt[i]))
        M[off[i]:off[i + 1], off[i]:off[i + 1]] += B + B.T
    M += np.diag(np.abs(M).sum(axis=1) + 1.0)
    return M, off


@pytest.mark.parametrize("shape", [(7,), (5, 4), (6, 6), (3, 3, 3), (4, 3, 5)])
def test_factor_count_equals_dense_cholesky_structure(shape):
    rng = np.random.default_rng(1)
    M, _ = _grid_matrix(shape, rng)
    order = bench._nd_order(shape)
    assert sorted(order.tolist()) == list(range(int(np.prod(shape))))
    L = np.linalg.cholesky(M[np.ix_(order, order)])
    assert int(np.count_nonzero(np.abs(L) > 1e-12)) == bench.grid_factor_nnz(shape)


def test_supernodal_count_equals_dense_cholesky_structure():
    rng = np.random.default_rng(2)
    shape = (3, 4)
    wt = rng.integers(1, 4, 12)
    M, off = _grid_matrix(shape, rng, wt)
    order = bench._nd_order(shape)
    perm = np.concatenate([np.arange(off[i], off[i + 1]) for i in order])
    L = np.linalg.cholesky(M[np.ix_(perm, perm)])
    assert int(np.count_nonzero(np.abs(L) > 1e-12)) == bench.grid_factor_nnz(shape, wt)


def test_block_shapes_cover_the_grid():
    shapes = bench._block_shapes((20, 17), 8)
    assert sum(int(np.prod(s)) * c for s, c in shapes.items()) == 20 * 17
    assert shapes == {(8, 8): 4, (8, 1): 2, (4, 8): 2, (4, 1): 1}
