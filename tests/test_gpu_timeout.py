"""Failure detection on the GPU without a fault: the bounded device-side
waits of the local solves (their factor-tile copies) end with
AMS_ERR_DEVICE_TIMEOUT when they run out, after the block has waited for
its own copies in flight, and leave the CUDA context usable.

ams_options.timeout_probe makes every local-solve block wait, within
spin_budget_cycles, on a barrier that nothing completes, so the timeout
path runs on purpose (for the one-RHS kernel and the several-RHS kernel).
"""

import numpy as np
import pytest

from oracle import OracleAMS, csr_to_scipy, pcg
from workloads import make_small_2d

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2606_04864_gb300 import AmsError, AmsSolver  # noqa: E402

TIMEOUT = 5


def _w(nrhs):
    return make_small_2d(side=96, bs=16, m=4, std=2.0, sigma=3.0, seed=81, nrhs=nrhs, rhs_kind="normal")


@pytest.mark.parametrize("nrhs", [1, 8])
def test_exhausted_wait_reports_timeout_and_context_survives(nrhs):
    w = _w(nrhs)
    A = csr_to_scipy(w.rowptr, w.colind, w.vals)
    f = w.rhs if nrhs > 1 else w.rhs[0]
    probe = AmsSolver(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m, precision="fp32_bf16",
                      autotune=False, spin_budget_cycles=20000, timeout_probe=True)
    with pytest.raises(AmsError) as e:
        probe.solve(f, rtol=1e-8)
    assert e.value.status == TIMEOUT
    with pytest.raises(AmsError) as e:
        probe.apply_preconditioner(f)
    assert e.value.status == TIMEOUT
    # the context is intact: no sticky CUDA error, device work still runs
    torch.cuda.synchronize()
    x = torch.ones(1000, device="cuda", dtype=torch.float64)
    assert float(x.sum()) == 1000.0
    # a handle with the default budget solves correctly on the same context
    good = AmsSolver(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m, precision="fp32_bf16", autotune=False)
    u, its, rel = good.solve(f, rtol=1e-8)
    u = np.atleast_2d(u)
    o = OracleAMS(A, w.part, w.nparts, w.m)
    for k in range(nrhs):
        ref = pcg(A, w.rhs[k], o.apply, rtol=1e-8)
        assert abs(int(its[k]) - ref.iters) <= 2
        assert np.linalg.norm(u[k] - ref.u) <= 1e-6 * np.linalg.norm(ref.u)
    # and the probe handle still fails cleanly on a second call
    with pytest.raises(AmsError) as e:
        probe.solve(f, rtol=1e-8)
    assert e.value.status == TIMEOUT


def test_budget_is_validated():
    w = _w(1)
    with pytest.raises(AmsError) as e:
        AmsSolver(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m, spin_budget_cycles=-1)
    assert e.value.status == 1
