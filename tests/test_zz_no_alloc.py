"""The allocation-free SpMV + dot entry point, through the C ABI.

It is for callers that cannot allocate device memory when they need the
product (for example while another library is capturing a CUDA graph).  It
is compared with the handle-based SpMV and with the host product of SciPy
on two calls in a row, since every call reuses the same fixed scratch
array inside the library.  This file is collected last so that a failure
here never hides the other tests.
"""

import ctypes

import numpy as np
import pytest
import scipy.sparse as sp

from workloads import make_small_2d, make_small_3d

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2606_04864_gb300 import AmsSolver, lib  # noqa: E402


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("make", [lambda: make_small_2d(side=200, bs=10, m=2, seed=90),
                                  lambda: make_small_3d(side=40, bs=8, m=2, seed=91)])
def test_noalloc_spmv_dot_matches_handle_spmv_twice(make):
    w = make()
    ref = AmsSolver(w.rowptr, w.colind, w.vals, w.part, w.nparts, 0, precision="fp64", coarse=False)
    A = sp.csr_matrix((w.vals, w.colind, w.rowptr), shape=(w.n, w.n))
    dev = torch.device("cuda")
    rowptr = torch.as_tensor(w.rowptr, device=dev)
    colind = torch.as_tensor(w.colind, device=dev)
    vals = torch.as_tensor(w.vals, device=dev)
    rng = np.random.default_rng(17)
    stream = torch.cuda.current_stream()
    for call in range(2):
        x_np = rng.standard_normal(w.n)
        x = torch.as_tensor(x_np, device=dev)
        y = torch.full((w.n,), float("nan"), dtype=torch.float64, device=dev)
        xy = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        st = lib().ams_csr_spmv_dot_noalloc(w.n, _p(rowptr), _p(colind), _p(vals), _p(x), _p(y), _p(xy),
                                            ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, lib().ams_last_error()
        torch.cuda.synchronize()
        y_ref = ref.spmv(x_np)
        y_np = y.cpu().numpy()
        assert np.abs(y_np - y_ref).max() <= 1e-13 * np.abs(y_ref).max(), call
        y_host = A @ x_np
        assert np.abs(y_np - y_host).max() <= 1e-13 * np.abs(y_host).max(), call
        d_ref = float(x_np @ y_host)
        assert abs(float(xy.item()) - d_ref) <= 1e-12 * abs(d_ref), call


def test_noalloc_rejects_sizes_beyond_its_scratch():
    dev = torch.device("cuda")
    dummy = torch.zeros(4, dtype=torch.float64, device=dev)
    idx = torch.zeros(4, dtype=torch.int64, device=dev)
    ci = torch.zeros(4, dtype=torch.int32, device=dev)
    st = lib().ams_csr_spmv_dot_noalloc(8_388_609, _p(idx), _p(ci), _p(dummy), _p(dummy), _p(dummy), _p(dummy),
                                        None)
    assert st == 1
    assert b"exceeds the scratch limit" in lib().ams_last_error()
