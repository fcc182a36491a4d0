"""Writes grf3d_128_apply_oracle.json: the CPU oracle's preconditioner
application z = M^{-1} r on the full-size 128^3 lognormal system (8^3-cell
subdomains, m = 6; 32 right-hand sides r drawn from
numpy.random.default_rng(128).standard_normal((32, n))), with the FP64
basis and with the basis rounded to bfloat16 (the coarse matrix formed from
the rounded basis), at 1024 seeded rows of every column.  Calls only the
oracle and the seeded workload generator; about half an hour of CPU time.

    python tests/golden/make_grf3d_128_apply_oracle.py
"""

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import OracleAMS, csr_to_scipy  # noqa: E402
from workloads import make_grf3d_128_rhs32  # noqa: E402


def main():
    w = make_grf3d_128_rhs32()
    A = csr_to_scipy(w.rowptr, w.colind, w.vals)
    r = np.random.default_rng(128).standard_normal((32, w.n))
    rows = np.sort(np.random.default_rng(2025).choice(w.n, size=1024, replace=False))
    out = {"workload": w.name, "n": w.n, "nnz": w.nnz, "rhs_seed": 128, "sample_idx": rows.tolist()}
    for rnd in (None, "bf16"):
        t0 = time.time()
        o = OracleAMS(A, w.part, w.nparts, w.m, basis_round=rnd)
        t1 = time.time()
        z = np.stack([o.apply(r[k])[rows] for k in range(32)])
        key = "fp64" if rnd is None else "bf16_basis"
        out[key] = {"z": z.tolist(), "ncoarse": int(o.Nc), "setup_s": round(t1 - t0, 1),
                    "apply_s": round(time.time() - t1, 1)}
        print(key, out[key]["ncoarse"], out[key]["setup_s"], out[key]["apply_s"], flush=True)
    with open(os.path.join(HERE, "grf3d_128_apply_oracle.json"), "w") as fh:
        json.dump(out, fh)


if __name__ == "__main__":
    main()
