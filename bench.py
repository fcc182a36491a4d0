"""Benchmark: AMS-preconditioned CG time-to-solution on one GB300.

Workload of the N=1 line (``--workload``, default ``grf3d_128_rhs32``): the
3-D lognormal Darcy system of 128^3 cells (log-std 3, Gaussian filter
sigma 6), 8^3-cell subdomains (4096), m = 6 eigenvectors each (N_c =
24,576), 32 right-hand sides iid N(0,1) solved as one multi-RHS solve, rtol
1e-8.  The mixed path (FP32 preconditioner apply, BF16 basis blocks,
flexible CG) is timed; the all-FP64 GPU path is reported beside it, and so
is the 1024^2 channelised system (one right-hand side) as a second
workload.  Other workloads: ``channels2d_1024``, ``grf3d_96`` (one
right-hand side) and ``batch48_uneven`` (48 systems of uneven size, 8
right-hand sides each, one batched handle).

A step is one complete solve (every kernel of the hot path, from the
right-hand sides resident in HBM to the solutions in HBM).  Setup is not
timed (it is reported).  The working set (matrix, factors, basis, coarse
inverse and vectors: several GB at 128^3 x 32) exceeds the 129 MB L2, so no
flush is needed between steps.

Roofline: the dominant kernel's algorithmic bytes per launch follow the
per-iteration byte model of the hot-path scope (each operand read once and
each output written once; local factors counted with their nested-
dissection fill, the coarse factor likewise), divided by its mean launch
time measured with CUDA events inside a real solve.  The bytes the library
actually stores for that kernel (band factor tiles, explicit coarse inverse
blocks) are reported beside them as ``stored_bytes_per_launch``.

Under torchrun every rank solves its own copy of the workload (weak
scaling, no collective on the data path); value is the slowest rank's
time.  ``--impl reference`` times the CPU oracle instead on a labelled
sample of the same workload (see --help).
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
WORKLOADS = ("grf3d_128_rhs32", "channels2d_1024", "grf3d_96", "batch48_uneven")

# Kernel behind each timed solve slot, for the ncu traffic lookup.
SLOT_KERNELS = {"local_solve_restrict": ("k_local_mma", "k_local_tma1", "k_local_tma"),
                "spmv_direction": ("k_spmv_dot",),
                "coarse_solve": ("k_coarse_mma", "k_coarse_gemm", "k_coarse_rows"),
                "prolong_update": ("k_prolong_update",)}


def _make(name):
    import workloads as W
    return {"grf3d_128_rhs32": W.make_grf3d_128_rhs32, "channels2d_1024": W.make_channels2d_1024,
            "grf3d_96": W.make_grf3d_96_adjoint, "batch48_uneven": W.make_batch48_uneven}[name]()


# ---------------------------------------------------------------------------
# algorithmic bytes (per-iteration byte model of the hot path)
# ---------------------------------------------------------------------------

def _nd_order(shape):
    """Geometric nested dissection of a box of grid cells: halve the longest
    axis, order both halves recursively, the middle plane (separator) last."""
    idx = np.arange(int(np.prod(shape))).reshape(shape)
    order = []

    def rec(lo, hi):
        sizes = [h - l for l, h in zip(lo, hi)]
        if min(sizes) <= 0:
            return
        box = tuple(slice(l, h) for l, h in zip(lo, hi))
        if max(sizes) <= 2 or int(np.prod(sizes)) <= 4:
            order.extend(idx[box].ravel().tolist())
            return
        ax = int(np.argmax(sizes))
        mid = lo[ax] + sizes[ax] // 2
        left_hi = list(hi)
        left_hi[ax] = mid
        right_lo = list(lo)
        right_lo[ax] = mid + 1
        rec(list(lo), left_hi)
        rec(right_lo, list(hi))
        s_lo, s_hi = list(lo), list(hi)
        s_lo[ax], s_hi[ax] = mid, mid + 1
        order.extend(idx[tuple(slice(l, h) for l, h in zip(s_lo, s_hi))].ravel().tolist())

    rec([0] * len(shape), list(shape))
    return np.asarray(order, dtype=np.int64)


def grid_factor_nnz(shape, weights=None) -> int:
    """Entries (diagonal included) of the Cholesky factor of a (2d+1)-point
    grid matrix on a box of cells, under the nested-dissection order above.
    With ``weights`` (C order over the cells) each cell is a supernode of
    that many unknowns, dense within and between coupled supernodes (the
    coarse matrix on the subdomain grid).  Symbolic factorisation: the
    elimination tree with path compression, then the row subtrees."""
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape))
    order = _nd_order(shape)
    wt = np.ones(n, dtype=np.int64) if weights is None else np.asarray(weights, dtype=np.int64).reshape(-1)
    wt = wt[order]                       # in elimination order
    idx = np.arange(n).reshape(shape)
    pos = np.empty(n, dtype=np.int64)
    pos[order] = np.arange(n)
    lower = [[] for _ in range(n)]
    for ax in range(len(shape)):
        a = np.moveaxis(idx, ax, 0)
        for x, y in zip(pos[a[:-1].ravel()], pos[a[1:].ravel()]):
            lower[max(x, y)].append(min(x, y))
    parent, anc = [-1] * n, [-1] * n
    for i in range(n):
        for k in lower[i]:
            j = k
            while anc[j] != -1 and anc[j] != i:
                nxt = anc[j]
                anc[j] = i
                j = nxt
            if anc[j] == -1:
                anc[j] = i
                parent[j] = i
    mark, tot = [-1] * n, 0
    for i in range(n):
        mark[i] = i
        tot += int(wt[i] * (wt[i] + 1) // 2)
        for k in lower[i]:
            j = k
            while mark[j] != i:
                mark[j] = i
                tot += int(wt[i] * wt[j])
                j = parent[j]
    return tot


def _block_shapes(shape, bs):
    """Distinct subdomain shapes of a regular block partition with counts."""
    per_axis = [[(bs, s // bs)] + ([(s % bs, 1)] if s % bs else []) for s in shape]
    out = {}

    def rec(ax, cur, cnt):
        if ax == len(shape):
            out[tuple(cur)] = out.get(tuple(cur), 0) + cnt
            return
        for ext, c in per_axis[ax]:
            if c:
                rec(ax + 1, cur + [ext], cnt * c)

    rec(0, [], 1)
    return out


def local_factor_nnz(w) -> int:
    """Sum over subdomains of nnz(L_i), nested-dissection fill."""
    return sum(cnt * grid_factor_nnz(sh) for sh, cnt in _block_shapes(w.shape, w.extra["bs"]).items())


def coarse_factor_nnz(w, m_i) -> int:
    """nnz(L_c) of the coarse Cholesky factor with nested-dissection fill:
    the subdomain grid (face-adjacent blocks couple in A_0), each subdomain
    a supernode of its m_i unknowns."""
    bshape = tuple((s + w.extra["bs"] - 1) // w.extra["bs"] for s in w.shape)
    return grid_factor_nnz(bshape, m_i)


def slot_bytes(systems, nrhs, prec="mixed"):
    """Algorithmic bytes per launch of each timed slot of the iteration (the
    library's slot order) for a list of (workload, m_i) systems solved
    together, FP32 preconditioner with BF16 basis ("mixed") or FP64.  Each
    operand read once and each output written once; the local factors and
    the coarse factor with nested-dissection fill (the coarse factor once
    per sweep)."""
    bF = 4 if prec == "mixed" else 8
    bP = 2 if prec == "mixed" else 8
    n = sum(w.n for w, _ in systems)
    nnz = sum(w.nnz for w, _ in systems)
    nc = sum(int(np.sum(m_i)) for _, m_i in systems)
    psi = sum(int(np.sum(_psi_entries(w, m_i))) for w, m_i in systems)
    lnz = sum(local_factor_nnz(w) for w, _ in systems)
    cnz = sum(coarse_factor_nnz(w, m_i) for w, m_i in systems)
    fused = nrhs <= 4
    # from 5 right-hand sides (stride 8) x += alpha p_old of the previous
    # iteration rides on the direction update; below, the prolongation does it
    xdir = nrhs > 4
    nv = n * nrhs
    return {
        # z (apply precision), p_old in; p, q out; x in and out when xdir; A
        # (values, columns, row pointers)
        "spmv_direction": 12 * nnz + 4 * (n + len(systems)) + (24 + bF + (16 if xdir else 0)) * nv,
        # factor once; r, q in; z_f, r_c out; basis rows
        "local_solve_restrict": bF * lnz + 16 * nv + bF * nv + bP * psi + bF * nc * nrhs,
        # forward sweep (and the backward one when separate): factor, r_c in, y out
        "coarse_solve": (bF * cnz + 2 * bF * nc * nrhs) * (1 if fused else 2),
        # (backward sweep when fused) e_c in, z_f, basis; r, q in; r out, z out
        # (apply precision); p, x in and x out unless xdir
        "prolong_update": (bF * cnz + bF * nc * nrhs if fused else 0) + bF * nc * nrhs + bF * nv + bP * psi
        + (24 + bF + (0 if xdir else 24)) * nv,
        "_nnz_local_factor_nd": lnz, "_nnz_coarse_factor_nd": cnz,
    }


def slot_fp64_flops(systems, nrhs):
    """FP64 floating-point operations per launch of each slot (an FMA counts
    two): the SpMV and its fused dot and direction update, the residual
    update the local solves form, and the prolongation's CG update and
    dots, with the x update on the direction update of the next iteration
    from 5 right-hand sides and on the prolongation below.  The
    preconditioner itself runs in FP32/TF32."""
    n = sum(w.n for w, _ in systems)
    nnz = sum(w.nnz for w, _ in systems)
    nv = n * nrhs
    xdir = nrhs > 4
    return {"spmv_direction": 2 * nnz * nrhs + (6 if xdir else 4) * nv,   # q = A p, p = z + beta p_old, p.q
            "local_solve_restrict": 2 * nv,                                # r' = r - alpha q
            "coarse_solve": 0,
            "prolong_update": (8 if xdir else 10) * nv}                    # r update; r.z, r.r, z.q; x


# FP64 peak (no measured figure exists for it): the nominal GB300 rate
FP64_PEAK_TFLOPS = 1.25


def default_m_i(w):
    """m_i = min(m, n_i) per subdomain of a regular block partition."""
    from workloads import block_partition
    part, nparts = block_partition(w.shape, w.extra["bs"])
    return np.minimum(w.m, np.bincount(part, minlength=nparts))


def _psi_entries(w, m_i):
    from workloads import block_partition
    part, nparts = block_partition(w.shape, w.extra["bs"])
    ni = np.bincount(part, minlength=nparts)
    return ni * np.asarray(m_i)


def kernel_text(path: str, kernel: str):
    """The definition of the `__global__` function `kernel` in `path`: from
    its name to the brace closing its body (None if not found)."""
    text = open(path, errors="replace").read()
    pos = 0
    while True:
        i = text.find(kernel + "(", pos)
        if i < 0:
            return None
        head = text[max(0, i - 400):i]
        g = head.rfind("__global__")
        if g >= 0 and ";" not in head[g:] and "}" not in head[g:]:
            break
        pos = i + 1
    j = text.find("{", i)
    depth = 0
    for k in range(j, len(text)):
        if text[k] == "{":
            depth += 1
        elif text[k] == "}":
            depth -= 1
            if depth == 0:
                return text[i:k + 1]
    return None


def kernel_hash(path: str, kernel: str):
    """First 16 hex digits of the SHA-256 of the kernel's definition text."""
    import hashlib
    t = kernel_text(path, kernel)
    return None if t is None else hashlib.sha256(t.encode()).hexdigest()[:16]


def _profiled_traffic(kernel: str, workload=None):
    """DRAM bytes per launch of `kernel` and the summary's workload from a
    committed ncu summary under profiles/, or None when no summary matches
    the kernel's current definition (the counters describe only the code
    they were taken from: the summary records the hash of the kernel's
    definition text, so edits elsewhere in its file do not void it)."""
    import glob
    import re
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path, errors="replace"):
            mt = re.match(r"traffic_bytes_per_launch: (\d+) kernel: (\S+) source: (\S+) kernel_sha256_16: ([0-9a-f]{16})"
                          r"(?: workload: (\S+))?", line.strip())
            if not mt or mt.group(2) != kernel:
                continue
            if workload is not None and mt.group(5) not in (None, workload):
                continue
            src = os.path.join(ROOT, mt.group(3))
            if not os.path.exists(src):
                continue
            if kernel_hash(src, kernel) == mt.group(4):
                return int(mt.group(1)), os.path.relpath(path, ROOT), mt.group(5)
    return None, None, None


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
# CPU oracle leg (labelled sample, measured, not scaled)
# ---------------------------------------------------------------------------

class OracleSample:
    """The CPU oracle, as it stands, on a labelled sample of the workload:
    a window of the same permeability field with the same generator,
    subdomain size, m and rtol, and the first right-hand sides of that
    window.  One step is the oracle's complete PCG solve of every sample
    right-hand side (setup separate, reported).  The value is the measured
    time of that sample; it is not scaled to the full workload (the
    oracle's cost is not linear in the size: its coarse solve is dense)."""

    SAMPLES = {   # workload: (window side, right-hand sides)
        "grf3d_128_rhs32": (32, 2),
        "channels2d_1024": (256, 1),
        "grf3d_96": (32, 1),
        "batch48_uneven": (0, 1),
    }

    def __init__(self, name: str):
        from oracle import OracleAMS, csr_to_scipy
        from workloads import channel_field, grf_logk, make_from_logk
        side, nrhs = self.SAMPLES[name]   # side 0: a member of the batch itself
        if name == "grf3d_128_rhs32":
            logk = grf_logk((128,) * 3, sigma=6.0, std=3.0, seed=3)[:side, :side, :side]
            self.w = make_from_logk(f"grf3d_128_window{side}", logk, 8, 6, rhs_kind="normal", nrhs=nrhs, seed=3)
            desc = f"{side}^3 window of the 128^3 field (8^3 blocks, m=6), {nrhs} of the N(0,1) right-hand sides"
        elif name == "channels2d_1024":
            logk = channel_field((1024, 1024), nchannels=200, kmax=1e6, seed=2)[:side, :side]
            self.w = make_from_logk(f"channels2d_1024_window{side}", logk, 32, 8)
            desc = f"{side}^2 window of the 1024^2 channel field (32^2 blocks, m=8), f = h^2"
        elif name == "grf3d_96":
            logk = grf_logk((96,) * 3, sigma=6.0, std=2.0, seed=5)[:side, :side, :side]
            self.w = make_from_logk(f"grf3d_96_window{side}", logk, 8, 6)
            desc = f"{side}^3 window of the 96^3 field (8^3 blocks, m=6), f = h^3"
        else:
            from workloads import make_batch48_uneven
            ws = make_batch48_uneven()
            self.w = min(ws, key=lambda x: x.n)
            self.w.rhs = self.w.rhs[:nrhs]
            desc = (f"the smallest of the 48 systems ({self.w.name}, {self.w.n} dofs, m={self.w.m}), "
                    f"{nrhs} of its 8 right-hand sides")
        self.A = csr_to_scipy(self.w.rowptr, self.w.colind, self.w.vals)
        t0 = time.perf_counter()
        self.o = OracleAMS(self.A, self.w.part, self.w.nparts, self.w.m)
        self.t_setup = time.perf_counter() - t0
        self.desc = desc

    def step(self):
        from oracle import pcg
        t0, c0 = time.perf_counter(), time.process_time()
        its = [pcg(self.A, self.w.rhs[k], self.o.apply, rtol=1e-8).iters for k in range(self.w.nrhs)]
        wall, cpu = time.perf_counter() - t0, time.process_time() - c0
        return wall, {"sample": self.desc, "n": self.w.n, "nparts": self.w.nparts, "nrhs": self.w.nrhs,
                      "iters": its, "setup_s": round(self.t_setup, 3), "cpu_s": round(cpu, 3)}, cpu / max(wall, 1e-9)


def run_reference(args):
    """--impl reference: the CPU oracle as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    smp = OracleSample(args.workload)
    for _ in range(args.warmup):
        smp.step()
    vals, detail, par = [], None, []
    for _ in range(args.steps):
        v, detail, p = smp.step()
        vals.append(v)
        par.append(p)
    v = float(np.median(vals))
    cores = max(1, int(round(float(np.median(par)))))
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample": detail["sample"], "sample_n": detail["n"],
                   "sample_nrhs": detail["nrhs"], "rtol": 1e-8,
                   "note": "oracle solve of a labelled window of the workload, measured, not scaled"},
        "cpu_baseline": {"value": v, "unit": "s", "cores": cores, "host_cpus": os.cpu_count(), "kind": "oracle",
                         "sample": json.dumps(detail)},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------

def _timed(fn, steps, stream, torch):
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    out = None
    for _ in range(steps):
        out = fn()
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / steps, out


def _second_workload(name, torch, stream):
    """Mixed and FP64 time-to-solution of a second workload (3 solves each)."""
    from paper_2606_04864_gb300 import AmsSolver
    w = _make(name)
    f = torch.as_tensor(w.rhs, device="cuda")
    out = {"workload": w.name, "n": w.n, "nrhs": w.nrhs}
    for prec in ("fp32_bf16", "fp64"):
        s = AmsSolver(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m, precision=prec, device=True)
        s.solve(f, rtol=1e-8)
        ms, (u, its, rel) = _timed(lambda: s.solve(f, rtol=1e-8), 3, stream, torch)
        out["mixed" if prec != "fp64" else "fp64"] = {"time_s": ms / 1e3, "iters": int(its.max()),
                                                      "setup_s": round(s.info()["setup_seconds"], 3)}
        s.close()
    out["mixed_speedup_vs_fp64"] = out["fp64"]["time_s"] / out["mixed"]["time_s"]
    s = AmsSolver(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m, precision="fp32_bf16", device=True,
                  two_grid_omega=-1.0)
    s.solve(f, rtol=1e-8)
    ms, (u, its, rel) = _timed(lambda: s.solve(f, rtol=1e-8), 3, stream, torch)
    out["two_grid_cycle"] = {"time_s": ms / 1e3, "iters": int(its.max()), "omega": s.info()["two_grid_omega"]}
    s.close()
    return out


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2606_04864_gb300 import AmsBatchedSolver, AmsSolver

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    batched = args.workload == "batch48_uneven"
    W = _make(args.workload)
    if batched:
        ws = W
        nrhs = ws[0].nrhs
        systems = [(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m) for w in ws]

        def build(prec, device):
            return AmsBatchedSolver(systems, precision=prec, device=device)

        rhs_host = np.concatenate([w.rhs.reshape(-1) for w in ws])
        f_dev = torch.as_tensor(rhs_host, device=dev)
        n_total = sum(w.n for w in ws)
        nnz_total = sum(w.nnz for w in ws)
        name = "batch48_uneven"
        cfg_extra = {"nsys": len(ws), "n": n_total, "nnz": nnz_total, "nrhs": nrhs,
                     "sizes": [w.n for w in ws]}

        def solve(s, f):
            return s.solve(f, nrhs, rtol=1e-8)
    else:
        w = W
        nrhs = w.nrhs

        def build(prec, device):
            return AmsSolver(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m, precision=prec, device=device)

        rhs_host = w.rhs
        f_dev = torch.as_tensor(w.rhs, device=dev)
        n_total = w.n
        name = w.name
        cfg_extra = {"n": w.n, "nnz": w.nnz, "nparts": w.nparts, "m": w.m, "nrhs": nrhs}

        def solve(s, f):
            return s.solve(f, rtol=1e-8)

    # one-time process costs (CUDA context, module loading, solver library
    # initialisation) on a tiny system first, so the setups below time only
    # their own work
    from workloads import make_small_2d
    t_first = time.perf_counter()
    tiny = make_small_2d(side=16, bs=8, m=2)
    AmsSolver(tiny.rowptr, tiny.colind, tiny.vals, tiny.part, tiny.nparts, tiny.m, precision="fp32_bf16",
              device=True).close()
    first_call_s = time.perf_counter() - t_first
    t_setup0 = time.perf_counter()
    mixed = build("fp32_bf16", True)
    setup_wall = time.perf_counter() - t_setup0
    info = mixed.info()
    if args.launch_shape and not batched:
        mixed.set_launch_shape(nrhs, **dict(zip(("bps_elem", "bps_sub", "depth", "nr", "l2mode", "l2keep"),
                                                (int(v) for v in args.launch_shape.split(",")))))
    for _ in range(args.warmup):
        u, its, rel = solve(mixed, f_dev)
    launches0 = mixed.info()["kernel_launches"]
    shape = mixed.launch_shape(nrhs)
    barrier()
    with ClockSampler(torch.cuda.current_device()) as clk:
        ms, (u, its, rel) = _timed(lambda: solve(mixed, f_dev), args.steps, stream, torch)
        barrier()
    launches = mixed.info()["kernel_launches"] - launches0
    ms_max = slowest_rank(ms, world, dev)

    # true residuals (host, FP64)
    from scipy.sparse import csr_matrix
    u_np = u.cpu().numpy()
    if batched:
        us = mixed.unpack(u_np, nrhs)
        true_rel = 0.0
        for i in range(0, len(ws), 7):
            A = csr_matrix((ws[i].vals, ws[i].colind, ws[i].rowptr), shape=(ws[i].n, ws[i].n))
            for k in range(nrhs):
                true_rel = max(true_rel, float(np.linalg.norm(ws[i].rhs[k] - A @ us[i][k])
                                               / np.linalg.norm(ws[i].rhs[k])))
    else:
        A = csr_matrix((w.vals, w.colind, w.rowptr), shape=(w.n, w.n))
        true_rel = max(float(np.linalg.norm(w.rhs[k] - A @ u_np[k]) / np.linalg.norm(w.rhs[k]))
                       for k in range(nrhs))

    # adjoint (a8), outside the timed region: L = |u|^2 / 2, dL/du = u
    adjoint = None
    if not batched:
        mixed.solve_adjoint(u, u, rtol=1e-8)
        nadj = max(1, min(args.steps, 3))
        ams, (lam, dv, its_adj) = _timed(lambda: mixed.solve_adjoint(u, u, rtol=1e-8), nadj, stream, torch)
        adjoint = {"time_s": ams / 1e3, "iters": int(np.max(its_adj)),
                   "loss": "L = |u|^2/2 (g = u); lambda = A^-1 g, dL/dA_ij = -lambda_i u_j on A's pattern"}

    # per-kernel device times inside one real solve (events around every
    # kernel on the library's stream, no graph capture)
    prof = mixed.profile_solve(f_dev, nrhs, rtol=1e-8) if batched else mixed.profile_solve(f_dev, rtol=1e-8)
    kern, roof = {}, None
    if prof is not None:
        if batched:   # m_i = min(m, n_i); the count agrees with the handle's coarse dimension
            sysm = [(x, default_m_i(x)) for x in ws]
            if sum(int(np.sum(mi)) for _, mi in sysm) != info["ncoarse"]:
                sysm = None
        else:
            sysm = [(w, mixed.coarse_basis()[0])]
        alg = slot_bytes(sysm, nrhs, "mixed") if sysm is not None else None
        f64 = slot_fp64_flops(sysm, nrhs) if sysm is not None else None
        peak_hbm, _ = _peaks()
        for pk in prof:
            if not pk["count"] or alg is None:
                continue
            avg = pk["ms"] / pk["count"]
            a = alg[pk["name"]]
            gbs = a / (avg * 1e-3) / 1e9 if avg > 0 else None
            tf = f64[pk["name"]] / (avg * 1e-3) / 1e12 if avg > 0 else None
            kern[pk["name"]] = {"ms_total": pk["ms"], "launches": pk["count"], "ms": avg,
                                "alg_bytes": a, "stored_bytes": pk["bytes"], "gbs": gbs,
                                "fp64_flops": f64[pk["name"]], "fp64_tflops": tf,
                                "hbm_frac": gbs / peak_hbm if gbs else None,
                                "fp64_frac": tf / FP64_PEAK_TFLOPS if tf else None}
        tot = sum(v["ms_total"] for v in kern.values())
        for v in kern.values():
            v["share"] = v["ms_total"] / tot if tot > 0 else None
        dom = max(kern, key=lambda k: kern[k]["ms_total"])
        traffic, traffic_src, traffic_wl, traffic_kernel = None, None, None, None
        for kname in SLOT_KERNELS.get(dom, ()):
            t, src, wl = _profiled_traffic(kname, args.workload)
            if t is not None and (wl is None or wl == args.workload):
                traffic, traffic_src, traffic_wl, traffic_kernel = t, src, wl, kname
                break
        peak, peak_kind = _peaks()
        kd = kern[dom]
        alu = (kd["fp64_frac"] or 0.0) > (kd["hbm_frac"] or 0.0)   # the binding roof
        roof = {
            "bound": "alu" if alu else "hbm", "kernel": dom,
            "achieved": kd["fp64_tflops"] if alu else kd["gbs"], "peak": FP64_PEAK_TFLOPS if alu else peak,
            "unit": "TFLOP/s (FP64)" if alu else "GB/s",
            "frac": kd["fp64_frac"] if alu else kd["hbm_frac"], "traffic": traffic,
            "hbm_frac": kd["hbm_frac"], "fp64_frac": kd["fp64_frac"],
            "traffic_source": traffic_src, "traffic_kernel": traffic_kernel,
            "peak_source": ("nominal GB300 FP64 1.25 TFLOP/s (about two FP64 FMAs per clock per SM at 2.07 GHz; "
                            "no measured FP64 peak)") if alu else f"{peak_kind} hbm_gbs (copy burst)",
            "timing": "CUDA events around every launch inside one profiled solve",
            "algorithmic_bytes_per_launch": kern[dom]["alg_bytes"],
            "stored_bytes_per_launch": kern[dom]["stored_bytes"],
            "byte_model": "operands once; local factors with nested-dissection fill "
                          f"({alg['_nnz_local_factor_nd']} entries), coarse factor likewise "
                          f"({alg['_nnz_coarse_factor_nd']} entries)",
        }

    # FP64 GPU path on the same systems (the "mixed vs FP64" half of the metric)
    fp64 = build("fp64", True)
    solve(fp64, f_dev)
    nfp = max(1, min(args.steps, 3))
    ms64, (u64, its64, _) = _timed(lambda: solve(fp64, f_dev), nfp, stream, torch)
    rel_mixed_vs_fp64 = float(torch.linalg.norm(u - u64) / torch.linalg.norm(u64))
    info64 = fp64.info()
    fp64.close()

    # multiplicative two-grid cycle (omega = 1 / lambda_max, estimated at setup)
    two_grid = None
    if not batched and not args.no_two_grid:
        tg = AmsSolver(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m, precision="fp32_bf16", device=True,
                       two_grid_omega=-1.0)
        solve(tg, f_dev)
        mtg, (utg, itg, _) = _timed(lambda: solve(tg, f_dev), nfp, stream, torch)
        ti = tg.info()
        two_grid = {"time_s": mtg / 1e3, "iters": int(np.max(itg)), "omega": ti["two_grid_omega"],
                    "lambda_max_estimate": ti["local_lambda_max"], "setup_s": round(ti["setup_seconds"], 3),
                    "u_rel_diff_vs_additive": float(torch.linalg.norm(utg - u) / torch.linalg.norm(u))}
        tg.close()

    # end to end through the public API with host buffers (pinned), copies timed
    host = build("fp32_bf16", False)
    f_pin = torch.empty(rhs_host.shape, dtype=torch.float64).pin_memory()
    f_pin.copy_(torch.as_tensor(rhs_host))
    f_np = f_pin.numpy()
    # the solution goes straight into pinned host memory
    u_np_pin = torch.empty(tuple(f_pin.shape), dtype=torch.float64).pin_memory().numpy()
    if not batched:
        solve_host = lambda s_, f_: s_.solve(f_, rtol=1e-8, out=u_np_pin)   # noqa: E731
    else:
        solve_host = lambda s_, f_: s_.solve(f_, nrhs, rtol=1e-8, out=u_np_pin)   # noqa: E731
    solve_host(host, f_np)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        uh, itsh, _ = solve_host(host, f_np)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps
    host.close()
    e2e_s = slowest_rank(e2e_s, world, dev)

    second = None
    if rank == 0 and world == 1 and args.workload == "grf3d_128_rhs32" and not args.no_second:
        second = _second_workload("channels2d_1024", torch, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        smp = OracleSample(args.workload)
        v, detail, par = smp.step()
        cpu = {"value": v, "unit": "s", "cores": max(1, int(round(par))), "host_cpus": os.cpu_count(),
               "kind": "oracle", "sample": json.dumps(detail),
               "note": "measured on the labelled sample, not scaled to the workload"}

    if rank == 0:
        config = {"workload": name, **cfg_extra,
                  "rtol": 1e-8, "precision": "fp32 apply + bf16 basis, flexible CG",
                  "iters": int(np.max(its)), "relres": float(np.max(rel)), "true_relres": true_rel,
                  "ncoarse": info["ncoarse"], "setup_s": round(info["setup_seconds"], 3),
                  "setup_wall_s": round(setup_wall, 3),
                  "first_call_s": round(first_call_s, 3),
                  "eig_s": round(info["eig_seconds"], 3), "eig_iterations": info["eig_iterations"],
                  "coarse_s": round(info["coarse_seconds"], 3),
                  "coarse_factor": {"s": round(info["coarse_factor_seconds"], 3),
                                    "gflop": round(info["coarse_factor_gflop"], 1),
                                    "gflop_per_s": round(info["coarse_factor_gflop"] /
                                                         max(info["coarse_factor_seconds"], 1e-9), 1)},
                  "l2": "working set > 129 MB L2 (no flush needed)",
                  "fp64": {"time_s": ms64 / 1e3, "iters": int(np.max(its64)),
                           "setup_s": round(info64["setup_seconds"], 3)},
                  "mixed_speedup_vs_fp64": ms64 / ms_max if ms_max > 0 else None,
                  "u_rel_diff_mixed_vs_fp64": rel_mixed_vs_fp64,
                  "launch_shape": {**shape, "source": "--launch-shape" if args.launch_shape else "autotuned"}}
        if adjoint is not None:
            config["adjoint"] = adjoint
        if two_grid is not None:
            config["two_grid_cycle"] = two_grid
        if kern:
            it_ms = sum(v["ms"] for v in kern.values())
            config["iteration_ms"] = it_ms
            config["iteration_gbs"] = sum(v["alg_bytes"] for v in kern.values()) / (it_ms * 1e-3) / 1e9
            config["kernels"] = {k: {"ms_per_launch": round(v["ms"], 5), "launches": v["launches"],
                                     "share": round(v["share"], 4), "alg_bytes": int(v["alg_bytes"]),
                                     "stored_bytes": int(v["stored_bytes"]),
                                     "gbs": round(v["gbs"], 1) if v["gbs"] else None,
                                     "hbm_frac": round(v["hbm_frac"], 3) if v["hbm_frac"] else None,
                                     "fp64_tflops": round(v["fp64_tflops"], 3) if v["fp64_tflops"] else None,
                                     "fp64_frac": round(v["fp64_frac"], 3) if v["fp64_frac"] else None}
                                 for k, v in kern.items()}
        if second is not None:
            config["channels2d_1024"] = second
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
            "config": config,
            "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": 8 * n_total * nrhs,
                    "d2h_bytes_per_step": 8 * n_total * nrhs + 12 * nrhs * (len(ws) if batched else 1)},
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
        }
        if roof is not None:
            line["roofline"] = roof
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    mixed.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_kernel_timing(args):
    """--kernel-timing: a smaller copy of the 3-D lognormal workload (side^3
    cells, same generator, 8^3 blocks, m = 6, nrhs N(0,1) right-hand sides;
    with --workload channels2d_1024 the 1024^2 channel workload itself)
    solved once on fixed default launch shapes, then every kernel slot
    launched directly (ams_time_kernel, outside any graph) a few times.  The
    small case for per-kernel ncu captures (-k <kernel> -s <n> -c <n>),
    which do not see kernels inside the solve's conditional graph."""
    import torch

    from paper_2606_04864_gb300 import AmsSolver
    from workloads import grf_logk, make_from_logk
    torch.cuda.set_device(0)
    if args.workload == "channels2d_1024":   # the one-right-hand-side workload itself
        w = _make("channels2d_1024")
    else:
        logk = grf_logk((args.side,) * 3, sigma=6.0, std=3.0, seed=3)
        w = make_from_logk(f"grf3d_{args.side}_rhs{args.nrhs}", logk, 8, 6, rhs_kind="normal", nrhs=args.nrhs,
                           seed=3)
    s = AmsSolver(w.rowptr, w.colind, w.vals, w.part, w.nparts, w.m, precision="fp32_bf16", device=True,
                  autotune=False)
    u, its, rel = s.solve(torch.as_tensor(w.rhs, device="cuda"), rtol=1e-8)
    out = {"workload": w.name, "n": w.n, "nrhs": w.nrhs, "iters": int(its.max()), "launch_shape": s.launch_shape(w.nrhs),
           "slots": {}}
    from paper_2606_04864_gb300._lib import KERNEL_NAMES
    for k, name in enumerate(KERNEL_NAMES):
        ms = [s.time_kernel(k, 3)[0] for _ in range(2)]
        out["slots"][name] = {"ms_per_launch": min(ms)}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-second", action="store_true", help="skip the second (1024^2) workload")
    ap.add_argument("--no-two-grid", action="store_true", help="skip the multiplicative two-grid cycle")
    ap.add_argument("--workload", default="grf3d_128_rhs32", choices=list(WORKLOADS),
                    help="grf3d_128_rhs32 (default, the headline line): 128^3 lognormal with 32 right-hand "
                         "sides; channels2d_1024: 1024^2 channelised Darcy; grf3d_96: 96^3 lognormal, one "
                         "right-hand side; batch48_uneven: 48 systems of uneven size, 8 right-hand sides each")
    ap.add_argument("--launch-shape", default="",
                    help="fix the mixed solver's launch shapes instead of autotuning them: "
                         "bps_elem,bps_sub,depth,nr,l2mode,l2keep (as reported in config.launch_shape); for "
                         "profiling one configuration under ncu, where autotuning timings are "
                         "distorted by the replays")
    ap.add_argument("--kernel-timing", action="store_true",
                    help="small 3-D case for per-kernel ncu captures: solve once, then launch every kernel slot "
                         "directly (see run_kernel_timing)")
    ap.add_argument("--side", type=int, default=96, help="--kernel-timing: cells per side")
    ap.add_argument("--nrhs", type=int, default=32, help="--kernel-timing: right-hand sides")
    args = ap.parse_args()
    if args.kernel_timing:
        return run_kernel_timing(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
