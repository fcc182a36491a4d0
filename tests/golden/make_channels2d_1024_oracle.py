"""Writes channels2d_1024_oracle.json: the CPU oracle's solve of the full-size
1024^2 channelised Darcy system (200 channels, k = 1e6, 32^2-cell subdomains,
m = 8, f = h^2), at rtol 1e-8 and 1e-13 (plain PCG, FP64 throughout).

Stored: iteration counts, solution norms, true relative residuals, the
oracle's own rtol-1e-8 error against its rtol-1e-13 solution (the
feasibility floor of the mixed-path tolerance) and the entries of both
solutions at 4096 seeded positions.  Calls only the oracle and the seeded
workload generator; about an hour of CPU time.

    python tests/golden/make_channels2d_1024_oracle.py
"""

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import OracleAMS, csr_to_scipy, pcg  # noqa: E402
from workloads import make_channels2d_1024  # noqa: E402


def main():
    t0 = time.time()
    w = make_channels2d_1024()
    A = csr_to_scipy(w.rowptr, w.colind, w.vals)
    o = OracleAMS(A, w.part, w.nparts, w.m)
    t_setup = time.time() - t0
    f = w.rhs[0]
    out = {"workload": w.name, "n": w.n, "nnz": w.nnz, "nparts": w.nparts, "m": w.m, "ncoarse": int(o.Nc),
           "setup_s": round(t_setup, 1)}
    sols = {}
    for rtol in (1e-8, 1e-13):
        t1 = time.time()
        res = pcg(A, f, o.apply, rtol=rtol)
        sols[rtol] = res.u
        out[f"rtol_{rtol:g}"] = {"iters": res.iters, "relres": res.relres, "true_relres": res.true_relres,
                                 "unorm": float(np.linalg.norm(res.u)), "solve_s": round(time.time() - t1, 1)}
    out["floor_rtol_1e-8_vs_1e-13"] = float(np.linalg.norm(sols[1e-8] - sols[1e-13]) / np.linalg.norm(sols[1e-13]))
    idx = np.sort(np.random.default_rng(2024).choice(w.n, size=4096, replace=False))
    out["sample_idx"] = idx.tolist()
    out["u_1e-8"] = sols[1e-8][idx].tolist()
    out["u_1e-13"] = sols[1e-13][idx].tolist()
    with open(os.path.join(HERE, "channels2d_1024_oracle.json"), "w") as fh:
        json.dump(out, fh)
    print(json.dumps({k: v for k, v in out.items() if not k.startswith(("sample", "u_"))}))


if __name__ == "__main__":
    main()
