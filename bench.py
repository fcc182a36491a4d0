"""Benchmark: AMS-preconditioned CG time-to-solution on one GB300.

Workload (N=1 line): the 2-D high-contrast Darcy system of 1024 x 1024
cells (200 seeded channels with k = 1e6 on k = 1), 32 x 32-cell
subdomains, m = 8 eigenvectors each, rtol 1e-8, one right-hand side; the
mixed path (FP32 preconditioner apply, BF16 basis blocks, flexible CG)
is timed, the all-FP64 GPU path is reported beside it.

A step is one complete solve (every kernel of the hot path, from the
right-hand side resident in HBM to the solution in HBM).  Setup is not
timed (it is reported).  The working set (~0.5 GB of matrix, factors,
basis, coarse inverse and vectors) exceeds the 129 MB L2, so no flush is
needed between steps.

Under torchrun every rank solves its own copy of the workload (weak
scaling, no collective on the data path); value is the slowest rank's
time.  ``--impl reference`` times the CPU oracle instead (see --help).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PCG time-to-solution at rtol 1e-8 (s), iters, HBM GB/s; mixed vs FP64"


# Kernel behind each timed solve step, for the ncu traffic lookup.
STEP_KERNELS = {"local_solve_restrict": "k_local_tma1"}


def _profiled_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from a committed ncu summary under
    profiles/, or None when no summary matches the kernel's current source
    (the counters describe only the source they were taken from)."""
    import glob
    import hashlib
    import re
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path, errors="replace"):
            m = re.match(r"traffic_bytes_per_launch: (\d+) kernel: (\S+) source: (\S+) sha256_16: ([0-9a-f]{16})",
                         line.strip())
            if not m or m.group(2) != kernel:
                continue
            src = os.path.join(ROOT, m.group(3))
            if not os.path.exists(src):
                continue
            if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] == m.group(4):
                return int(m.group(1)), os.path.relpath(path, ROOT)
    return None, None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"ams_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def slowest_rank(value: float, world: int, device=None) -> float:
    """Max over ranks of a per-rank time (the whole job ends with the slowest
    replica).  Uses whatever process group is initialised (NCCL on GPUs,
    gloo in the CPU tests)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# CPU oracle leg (bounded sample)
# ---------------------------------------------------------------------------

class OracleSample:
    """The CPU oracle on a bounded sample of the workload: a crop of the same
    field with the same generator, subdomain size, m and rtol.  Its
    per-iteration, per-dof solve time is scaled to the full workload's size
    and iteration count (the oracle's cost per iteration is linear in n)."""

    def __init__(self, full, crop: int = 256):
        from oracle import OracleAMS, csr_to_scipy
        from workloads import make_from_logk
        self.full = full
        logk = full.logk[:crop, :crop]
        self.w = make_from_logk(f"crop{crop}", logk, full.extra["bs"], full.m)
        self.A = csr_to_scipy(self.w.rowptr, self.w.colind, self.w.vals)
        t0 = time.perf_counter()
        self.o = OracleAMS(self.A, self.w.part, self.w.nparts, self.w.m)
        self.t_setup = time.perf_counter() - t0
        self.crop = crop

    def step(self, iters_full: int = 0):
        from oracle import pcg
        t0 = time.perf_counter()
        res = pcg(self.A, self.w.rhs[0], self.o.apply, rtol=1e-8)
        t_solve = time.perf_counter() - t0
        its = iters_full if iters_full > 0 else res.iters
        est = t_solve / max(res.iters, 1) / self.w.n * self.full.n * its
        detail = {
            "crop": f"{self.crop}x{self.crop} window of the same field ({self.w.n} dofs, "
                    f"{self.w.nparts} subdomains, m={self.w.m})",
            "crop_setup_s": round(self.t_setup, 3), "crop_solve_s": round(t_solve, 4),
            "crop_iters": res.iters,
            "scaled_to": f"{self.full.n} dofs x {its} iterations",
        }
        return est, detail


def run_reference(args):
    """--impl reference: the CPU oracle as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from workloads import make_channels2d_1024
    full = make_channels2d_1024()
    cores = os.cpu_count()
    smp = OracleSample(full, crop=args.ref_crop)
    for _ in range(args.warmup):
        smp.step(args.ref_iters)
    vals, detail = [], None
    for _ in range(args.steps):
        est, detail = smp.step(args.ref_iters)
        vals.append(est)
    v = float(np.median(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": full.name, "n": full.n, "nnz": full.nnz, "nparts": full.nparts, "m": full.m,
                   "rtol": 1e-8},
        "cpu_baseline": {"value": v, "unit": "s", "cores": cores, "kind": "oracle",
                         "sample": json.dumps(detail)},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------

def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2606_04864_gb300 import AmsSolver
    from workloads import make_channels2d_1024

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    from workloads import make_grf3d_128_rhs32, make_grf3d_96_adjoint
    w = {"channels2d_1024": make_channels2d_1024, "grf3d_128_rhs32": make_grf3d_128_rhs32,
         "grf3d_96": make_grf3d_96_adjoint}[args.workload]()
    f_dev = torch.as_tensor(w.rhs, device=dev)
    mixed = AmsSolver(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m, precision="fp32_bf16",
                      device=True)
    info = mixed.info()
    stream = torch.cuda.current_stream()
    if args.launch_shape:
        mixed.set_launch_shape(w.nrhs, **dict(zip(("bps_elem", "bps_sub", "depth", "nr", "l2mode", "l2keep"),
                                                  (int(v) for v in args.launch_shape.split(",")))))

    # warm-up
    for _ in range(args.warmup):
        u, its, rel = mixed.solve(f_dev, rtol=1e-8)
    launches0 = mixed.info()["kernel_launches"]
    shape = mixed.launch_shape(w.nrhs)
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            u, its, rel = mixed.solve(f_dev, rtol=1e-8)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = mixed.info()["kernel_launches"] - launches0
    ms_max = slowest_rank(ms, world, dev)
    u_np = u.cpu().numpy()
    from scipy.sparse import csr_matrix
    A = csr_matrix((w.vals, w.colind, w.rowptr), shape=(w.n, w.n))
    true_rel = max(float(np.linalg.norm(w.rhs[k] - A @ u_np[k]) / np.linalg.norm(w.rhs[k]))
                   for k in range(w.nrhs))

    # adjoint (a8), outside the timed region: for L = |u|^2 / 2, dL/du = u;
    # lambda = A^{-1} u by the same preconditioned CG, then dL/dA on A's pattern
    lam, dv, its_adj = mixed.solve_adjoint(u, u, rtol=1e-8)
    torch.cuda.synchronize()
    ea0 = torch.cuda.Event(enable_timing=True)
    ea1 = torch.cuda.Event(enable_timing=True)
    nadj = max(1, min(args.steps, 3))
    ea0.record(stream)
    for _ in range(nadj):
        lam, dv, its_adj = mixed.solve_adjoint(u, u, rtol=1e-8)
    ea1.record(stream)
    torch.cuda.synchronize()
    adjoint = {"time_s": ea0.elapsed_time(ea1) / nadj / 1e3, "iters": int(np.max(its_adj)),
               "loss": "L = |u|^2/2 (g = u); lambda = A^-1 g, dL/dA_ij = -lambda_i u_j on A's pattern"}

    # per-kernel device times measured inside a real solve: the library
    # records a CUDA event pair around every kernel on its stream during one
    # profiled solve (no graph capture) right after the timed region
    prof = mixed.profile_solve(f_dev, rtol=1e-8)
    kern = {}
    for pk in prof:
        name = pk["name"]
        avg = pk["ms"] / pk["count"] if pk["count"] else 0.0
        kern[name] = {"ms_total": pk["ms"], "launches": pk["count"], "ms": avg, "bytes": pk["bytes"],
                      "gbs": pk["bytes"] / (avg * 1e-3) / 1e9 if avg > 0 else None}
    tot = sum(v["ms_total"] for v in kern.values())
    for v in kern.values():
        v["share"] = v["ms_total"] / tot if tot > 0 else None
    dom = max(kern, key=lambda n: kern[n]["ms_total"])
    traffic, traffic_src = (None, None)
    if args.workload == "channels2d_1024" and dom in STEP_KERNELS:
        traffic, traffic_src = _profiled_traffic(STEP_KERNELS[dom])
    peak, peak_kind = _peaks()
    iter_bytes = sum(v["bytes"] for v in kern.values())
    it_ms = sum(v["ms"] for v in kern.values())

    # FP64 GPU path on the same system (the "mixed vs FP64" half of the metric)
    fp64 = AmsSolver(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m, precision="fp64", device=True)
    u64, its64, _ = fp64.solve(f_dev, rtol=1e-8)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    nfp = max(1, min(args.steps, 3))
    e0.record(stream)
    for _ in range(nfp):
        u64, its64, _ = fp64.solve(f_dev, rtol=1e-8)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1) / nfp
    rel_mixed_vs_fp64 = float(torch.linalg.norm(u - u64) / torch.linalg.norm(u64))
    info64 = fp64.info()
    fp64.close()

    # end to end through the public API with host buffers (pinned), copies timed
    host = AmsSolver(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m, precision="fp32_bf16", device=False)
    f_pin = torch.empty((w.nrhs, w.n), dtype=torch.float64).pin_memory()
    f_pin.copy_(torch.as_tensor(w.rhs))
    f_np = f_pin.numpy()
    host.solve(f_np, rtol=1e-8)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        uh, itsh, _ = host.solve(f_np, rtol=1e-8)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps
    host.close()
    e2e_s = slowest_rank(e2e_s, world, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "channels2d_1024":
        smp = OracleSample(w)
        est, detail = smp.step(int(its[0]))
        cpu = {"value": est, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": json.dumps(detail)}

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": ms_max / 1e3,
            "unit": "s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_max,
            "higher_is_better": False,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64+f32",
            "data": "synthetic",
            "config": {
                "workload": w.name, "n": w.n, "nnz": w.nnz, "nparts": w.nparts, "m": w.m, "nrhs": w.nrhs,
                "rtol": 1e-8, "precision": "fp32 apply + bf16 basis, flexible CG",
                "iters": int(its.max()), "relres": float(rel.max()), "true_relres": true_rel,
                "ncoarse": info["ncoarse"], "setup_s": round(info["setup_seconds"], 3),
                "eig_s": round(info["eig_seconds"], 3), "eig_iterations": info["eig_iterations"],
                "l2": "working set > 129 MB L2 (no flush needed)",
                "fp64": {"time_s": ms64 / 1e3, "iters": int(its64.max()),
                         "setup_s": round(info64["setup_seconds"], 3)},
                "mixed_speedup_vs_fp64": ms64 / ms_max if ms_max > 0 else None,
                "adjoint": adjoint,
                "launch_shape": {**shape, "source": "--launch-shape" if args.launch_shape else "autotuned"},
                "u_rel_diff_mixed_vs_fp64": rel_mixed_vs_fp64,
                "iteration_ms": it_ms, "iteration_gbs": iter_bytes / (it_ms * 1e-3) / 1e9,
                "kernels": {n: {"ms_per_launch": round(v["ms"], 5), "launches": v["launches"],
                                "share": round(v["share"], 4),
                                "gbs": round(v["gbs"], 1) if v["gbs"] else None}
                            for n, v in kern.items()},
            },
            "roofline": {
                "bound": "hbm", "kernel": dom,
                "achieved": kern[dom]["gbs"], "peak": peak, "unit": "GB/s",
                "frac": kern[dom]["gbs"] / peak, "traffic": traffic,
                "traffic_source": traffic_src,
                "peak_source": f"{peak_kind} hbm_gbs (copy burst)",
                "timing": "CUDA events around every launch inside one profiled solve",
                "algorithmic_bytes_per_launch": kern[dom]["bytes"],
            },
            "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": 8 * w.n * w.nrhs,
                    "d2h_bytes_per_step": 8 * w.n * w.nrhs + 12 * w.nrhs},
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    mixed.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="channels2d_1024",
                    choices=["channels2d_1024", "grf3d_128_rhs32", "grf3d_96"],
                    help="channels2d_1024 (default, the headline line): 1024^2 channelised Darcy; "
                         "grf3d_128_rhs32: 128^3 lognormal with 32 right-hand sides; grf3d_96: 96^3 "
                         "lognormal, one right-hand side")
    ap.add_argument("--launch-shape", default="",
                    help="fix the mixed solver's launch shapes instead of autotuning them: "
                         "bps_elem,bps_sub,depth,nr,l2mode,l2keep (as reported in config.launch_shape); for "
                         "profiling one configuration under ncu, where autotuning timings are "
                         "distorted by the replays")
    ap.add_argument("--ref-crop", type=int, default=256, help="oracle sample: crop side (cells)")
    ap.add_argument("--ref-iters", type=int, default=0,
                    help="oracle sample: iteration count of the full solve (0: the crop's own count)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
