"""The checking build (libams_debug.so, -DAMS_DEBUG) on the GPU: its
self-test records the planted check failure (site 99, a kernel that fails a
check without touching memory), and solves through every checked kernel
(SpMV, local solves with 1 and 32 right-hand sides, coarse products,
prolongation, permutations, batched systems of mixed band widths, the
adjoint) raise no check and match the oracle as the release build does.

Runs in a child process with AMS_LIBRARY=debug, so that the release and
checking libraries are never loaded into one process."""

import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import ctypes, json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2606_04864_gb300._build import build
build(debug=True)
from paper_2606_04864_gb300._lib import lib, LIB_PATH
from paper_2606_04864_gb300 import AmsSolver, AmsBatchedSolver
from oracle import OracleAMS, csr_to_scipy, pcg
from workloads import make_small_2d, make_small_3d
out = {"lib": LIB_PATH}
site = ctypes.c_int32(0)
assert lib().ams_debug_selftest(ctypes.byref(site)) == 0
out["selftest_site"] = site.value
w = make_small_2d(side=45, bs=10, m=3, std=2.0, sigma=3.0, seed=31, ny=37)
A = csr_to_scipy(w.rowptr, w.colind, w.vals)
o = OracleAMS(A, w.part, w.nparts, w.m)
o_apply = {"fp64": o, "fp32_bf16": OracleAMS(A, w.part, w.nparts, w.m, basis_round="bf16")}
f = np.random.default_rng(5).standard_normal((32, w.n))
errs = {}
for prec in ("fp64", "fp32_bf16"):
    s = AmsSolver(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m, precision=prec)
    for nrhs in (1, 32):
        u, its, rel = s.solve(f[:nrhs], rtol=1e-8)
        u = np.atleast_2d(u)
        e = 0.0
        for k in range(0, nrhs, 7):
            ref = pcg(A, f[k], o.apply, rtol=1e-8)
            e = max(e, float(np.linalg.norm(u[k] - ref.u) / np.linalg.norm(ref.u)))
        errs[f"{prec}_{nrhs}"] = e
    z = np.atleast_2d(s.apply_preconditioner(f[:4]))
    za = o_apply[prec].apply(f[0])
    errs[f"{prec}_apply"] = float(np.abs(z[0] - za).max() / np.abs(za).max())
    y = np.atleast_2d(s.spmv(f[:2]))
    errs[f"{prec}_spmv"] = float(np.abs(y[1] - A @ f[1]).max() / np.abs(A @ f[1]).max())
    if prec == "fp64":
        lam, dv, _ = s.solve_adjoint(f[:1], np.atleast_2d(s.solve(f[:1], rtol=1e-8)[0]))
        ref = pcg(A, f[0], o.apply, rtol=1e-8)
        errs["adjoint"] = float(np.linalg.norm(np.atleast_2d(lam)[0] - ref.u) / np.linalg.norm(ref.u))
ws = [make_small_2d(side=40, bs=8, m=4, std=2.0, seed=53), make_small_3d(side=16, bs=8, m=6, std=2.5, seed=54)]
b = AmsBatchedSolver([(x.rowptr, x.colind, x.vals, x.part, x.nparts, x.m) for x in ws], precision="fp32_bf16")
rhs = [np.random.default_rng(80 + i).standard_normal((8, x.n)) for i, x in enumerate(ws)]
u, its, rel = b.solve(b.pack(rhs), 8, rtol=1e-8)
us = b.unpack(u, 8)
e = 0.0
for i, x in enumerate(ws):
    Ax = csr_to_scipy(x.rowptr, x.colind, x.vals)
    ox = OracleAMS(Ax, x.part, x.nparts, x.m)
    ref = pcg(Ax, rhs[i][3], ox.apply, rtol=1e-8)
    e = max(e, float(np.linalg.norm(us[i][3] - ref.u) / np.linalg.norm(ref.u)))
errs["batched_mixed_band"] = e
out["errs"] = errs
print("RESULT " + json.dumps(out), flush=True)
"""


def test_checking_build_selftest_and_solves():
    env = dict(os.environ, AMS_LIBRARY="debug")
    p = subprocess.run([sys.executable, "-c", CHILD, ROOT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1500)
    assert p.returncode == 0, p.stdout[-3000:] + p.stderr[-3000:]
    line = [x for x in p.stdout.splitlines() if x.startswith("RESULT ")][-1]
    out = json.loads(line[len("RESULT "):])
    print(out)
    assert out["lib"].endswith("libams_debug.so")
    assert out["selftest_site"] == 99
    e = out["errs"]
    for k, v in e.items():
        tol = 1e-10 if k.startswith("fp64") or k == "adjoint" else (2e-5 if k.endswith("apply") else 1e-6)
        if k.endswith("spmv"):
            tol = 1e-13
        assert v <= tol, (k, v)


def test_release_build_selftest_reports_checks_compiled_out():
    import ctypes
    from paper_2606_04864_gb300._lib import LIB_PATH, lib
    if os.environ.get("AMS_LIBRARY") == "debug":  # pragma: no cover
        pytest.skip("this process runs the checking build")
    assert LIB_PATH.endswith("libams.so")
    site = ctypes.c_int32(-1)
    assert lib().ams_debug_selftest(ctypes.byref(site)) == 0
    assert site.value == 0
