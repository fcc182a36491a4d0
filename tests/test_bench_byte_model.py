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


def test_kernel_text_isolates_the_definition(tmp_path):
    """The traffic of a committed ncu summary is trusted only while the
    captured kernel's own definition is unchanged: its text runs from the
    name after `__global__` to the brace closing the body, launches and
    other functions of the file are not part of it."""
    src = tmp_path / "k.cu"
    body = (
        "template <int LD>\n__global__ void __launch_bounds__(256)\n"
        "k_demo(const double* x, double* y) {\n    if (x) { y[0] = x[0]; }\n}\n"
    )
    other = "void launch_demo() { k_demo<8><<<1, 1>>>(nullptr, nullptr); }\n"
    src.write_text("// header\n" + body + other)
    t = bench.kernel_text(str(src), "k_demo")
    assert t.startswith("k_demo(const double* x") and t.endswith("}") and "launch_demo" not in t
    h0 = bench.kernel_hash(str(src), "k_demo")
    src.write_text("// header changed\n" + body + other.replace("8", "16"))
    assert bench.kernel_hash(str(src), "k_demo") == h0          # edits elsewhere: same hash
    src.write_text("// header\n" + body.replace("y[0] = x[0]", "y[0] = 2 * x[0]") + other)
    assert bench.kernel_hash(str(src), "k_demo") != h0          # the kernel changed: new hash
    assert bench.kernel_text(str(src), "k_missing") is None


def test_committed_traffic_summaries_name_existing_kernels():
    """Every traffic line under profiles/ names a kernel that the named
    source defines (a summary can lapse, but not point at nothing)."""
    import glob
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    seen = 0
    for path in glob.glob(os.path.join(root, "profiles", "*.md")):
        for line in open(path):
            m = re.match(r"traffic_bytes_per_launch: \d+ kernel: (\S+) source: (\S+) kernel_sha256_16: [0-9a-f]{16}",
                         line.strip())
            if m:
                seen += 1
                assert bench.kernel_text(os.path.join(root, m.group(2)), m.group(1)) is not None, line
    assert seen > 0
