#!/usr/bin/env python
"""Parameter-sweep benchmark of the SPAI / SPAI-update / block-GMRES hot path on one GPU.

One step = one parameter sweep of the 3D 64^3 7-point workload (n = 262,144):
20 parameters p ~ U[0.1, 1] (sorted) x shifts s in {0.5, 1, 2} = 60 systems
A(p, s) = s^2 M + s D(p) + K(p), D = 0.05 M + 0.01 K(p), K(p) = K0 + p K1.  Per shift:
assemble + SPAI build at the first p and block-GMRES(50) solve, then for the other 19 p:
assemble + SPAI update (first approach of Table 1) + solve.  B = n x 8, N(0,1), tol 1e-8
on every column's true residual, FP64 throughout.  value = solves/s over the timed steps.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun each rank runs its own sweep on its own GPU (independent systems, no
collective; weak scaling) and rank 0 prints one JSON line.  ``--impl reference`` times the
CPU oracle (test infrastructure) on a bounded sample of the same workload instead.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "param-sweep solves/s to residual 1e-8, served vs plain FP64; HBM %; p99 latency"
UNIT = "solves/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=64)
    ap.add_argument("--nparams", type=int, default=20)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    # host threads (each with its own stream and context) sharing a shift's independent solves
    ap.add_argument("--workers", type=int, default=4)
    # single-kernel case (for profiler captures): H = V^T W or W -= V H at n = side^3, s = 8
    ap.add_argument("--kernel", default=None, choices=["dot", "update", "columns", "spmm32", "spmm"])
    ap.add_argument("--columns-workload", default="batched2d", choices=["batched2d", "sweep3d", "adaptive3d"],
                    help="--kernel columns: the batched 2D systems (FP32), one FP64 SPAI of the 3D sweep, "
                         "or one adaptive SPAI of the 3D sweep's matrix (--side sets the grid)")
    ap.add_argument("--columns-prec", default="fp64", choices=["fp64", "fp32"],
                    help="factor precision of the sweep3d column case")
    ap.add_argument("--columns-normal", action="store_true",
                    help="column case: solve the column problems by their normal equations (SPAI_LS_NORMAL)")
    ap.add_argument("--columns-variant", type=int, default=0,
                    help="pin this column-kernel variant code for the 25 x 7 tiles of the sweep3d column case")
    ap.add_argument("--nblk", type=int, default=16)
    ap.add_argument("--orth", default="tensor", choices=["tensor", "fp64"])
    # serving: Poisson arrivals over a pool of 16 3D 7-point grids (sides 24-96)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-only", action="store_true")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-fifo-seconds", type=float, default=2.0)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-rates", default="300,400", help="further offered rates of the serving workload")
    ap.add_argument("--serve-rate-seconds", type=float, default=4.0)
    ap.add_argument("--no-served-sweep", action="store_true")
    ap.add_argument("--gcro-kmax", type=int, default=16, help="recycled columns per shift of the block GCRO leg")
    # large workload: 3D 128^3 27-point grid, 16 RHS, BF16-stored SPAI, update vs rebuild
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--large-only", action="store_true")
    ap.add_argument("--large-side", type=int, default=128)
    ap.add_argument("--large-params", type=int, default=3)
    # batched workload: 256 independent 2D 5-point systems, sides 48-256
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-adaptive", action="store_true")
    ap.add_argument("--batched-only", action="store_true")
    ap.add_argument("--batched-systems", type=int, default=256)
    ap.add_argument("--batched-workers", type=int, default=8)
    return ap.parse_args()


def workload_config(w, nnz):
    return {
        "workload": f"3d-{w.dims[0]}^3-7pt parameter sweep: {len(w.params)} p x {len(w.shifts)} s, "
                    f"{w.B.shape[1]} RHS, SPAI(pattern A) build per shift + updates (Table 1 first "
                    f"approach), block GMRES({w.restart}), tol {w.tol:g}, FP64",
        "n": w.n, "nnz": int(nnz), "systems_per_step": len(w.params) * len(w.shifts),
        "nrhs": int(w.B.shape[1]), "restart": w.restart,
        "l2": "no flush: the per-solve working set (Krylov basis, 0.86 GB at n=262144) exceeds L2",
    }


# ------------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------------------ rooflines
def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    pk = json.load(open(path)) if os.path.exists(path) else {}
    src = "measured" if pk else "fallback"
    return (pk.get("hbm_gbs", 6800.0), pk.get("bf16_tflops", 1900.0),
            pk.get("bf16_tflops_sustained", 1700.0), src)


# FP64 ALU peak from unit counts and clock: 152 SMs x 2 FP64 FMA lanes/clk x 2 flop x 2.07 GHz
FP64_NOMINAL_TFLOPS = 152 * 4 * 2070e6 / 1e12
# FP32 ALU peak from unit counts and clock: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2070e6 / 1e12
# one FP64-accurate product of the digit kernels costs 43 BF16 digit-pair products
DIGIT_PRODUCTS = 43
# how each kernel family computes: FP64 ALUs, tensor cores (digit products), or neither
FAMILY_UNIT = {
    "block_dot_tc": "tensor", "block_update_tc": "tensor", "to_fixed": "none",
    "axpy": "none", "gather_csc": "none", "small_dense": "latency", "arnoldi_ls": "latency",
    "backsolve": "latency", "spmm32_A": "fp32", "spmm32_P": "fp32", "scale_rows32": "fp32", "round_f32": "none",
}
# DRAM bytes per launch, (a * blocks + b) * n * s, where blocks = algorithmic bytes per launch
# / (8 n s) (the Gram product: basis blocks + W; the update: basis blocks + W read and
# written): a = 8 B per entry, b fitted to one ncu capture of the kernel at n = 262,144,
# s = 8, 16 basis blocks (read + write bytes; summarised under profiles/).  A family is
# left out (traffic null) while its kernel has changed since its capture.
NCU_TRAFFIC = {
    "block_dot_tc": (8.0, (296.053e6 + 3.258e6) / 2097152 - 8.0 * 17),
    "block_update_tc": (8.0, (285.268e6 + 11.305e6) / 2097152 - 8.0 * 18),
}


def roofline_entry(f, n, s, fp64_probe=None, fp32_probe=None, unit=None):
    """Binding roof of one kernel family: max(bytes / HBM, flops / compute peak).

    Bytes and flops are the algorithmic figures of the method (FP64 operands), credited per
    launch by the library's profiler.  Compute peak: the FP64 ALUs for FP64 kernels, the
    FP32 ALUs for FP32 kernels (`unit` overrides the family's default, e.g. the column
    problems of an FP32 build), the BF16 tensor peak / 43 for the digit-product kernels
    (FP64-equivalent flops).  The FMA probes' measured rates are quoted beside the derived
    peaks."""
    hbm, bf16, bf16_sus, src = _peaks()
    unit = unit or FAMILY_UNIT.get(f["name"], "fp64")
    launches = max(f["launches"], 1)
    sec = f["ms"] * 1e-3
    out = {"kernel": f["name"], "launches": f["launches"], "avg_launch_ms": f["ms"] / launches,
           "algorithmic_bytes_per_launch": f["bytes"] / launches,
           "algorithmic_flops_per_launch": f["flops"] / launches}
    if unit == "latency" or sec <= 0:
        out.update({"bound": "latency", "achieved": None, "peak": None, "unit": None, "frac": None,
                    "traffic": None})
        return out
    cpeak = {"fp64": FP64_NOMINAL_TFLOPS, "fp32": FP32_NOMINAL_TFLOPS,
             "tensor": bf16_sus / DIGIT_PRODUCTS}.get(unit, 0.0)
    t_hbm = f["bytes"] / (hbm * 1e9)
    t_alu = f["flops"] / (cpeak * 1e12) if cpeak > 0 else 0.0
    if t_hbm >= t_alu:
        ach = f["bytes"] / sec / 1e9
        out.update({"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                    "peak_source": f"{src} copy bandwidth"})
    else:
        ach = f["flops"] / sec / 1e12
        out.update({"bound": "alu", "achieved": ach, "peak": cpeak, "unit": "TFLOP/s", "frac": ach / cpeak,
                    "peak_source": ("derived: 152 SM x 256 FP32 flop/clk x 2.07 GHz"
                                    + (f"; FP32 FMA probe measured {fp32_probe:.1f} TFLOP/s in this run"
                                       if fp32_probe else "") if unit == "fp32" else
                                    "derived: 152 SM x 4 FP64 flop/clk x 2.07 GHz"
                                    + (f"; FMA probe measured {fp64_probe:.3f} TFLOP/s in this run"
                                       if fp64_probe else ""))})
    # the compute side's fraction as well, whichever roof binds (an FP32 kernel near the
    # ridge can be HBM-bound by its algorithmic bytes and still far from the FP32 ALU peak)
    out["alu_frac"] = f["flops"] / sec / 1e12 / cpeak if cpeak > 0 else None
    out["traffic"] = None
    if f["name"] in NCU_TRAFFIC and f["bytes"] > 0:
        a, b = NCU_TRAFFIC[f["name"]]
        # blocks per launch recovered from the algorithmic bytes (8 B per element per block)
        blocks = f["bytes"] / launches / (8.0 * n * s)
        out["traffic"] = (a * blocks + b) * n * s
    return out


def run_columns_case(args):
    """The batched build on its own (`--kernel columns`): spai_build_batch of the
    many-small-systems workload (`--batched-systems` 2D 5-point systems, FP32 factors),
    warm-up builds (the first one tunes the team sizes) then timed builds, with the
    library's per-phase device times."""
    import torch
    import synth
    import paper_1809_06574_gb300 as sg
    if args.columns_workload in ("sweep3d", "adaptive3d"):  # one SPAI of the sweep's first system
        ws = [synth.grid3d_7pt(side=args.side, nparams=args.nparams)]
        kinds = [sg.PATTERN_A | (sg.PREC_FP32 if args.columns_prec == "fp32" else 0)]
        if args.columns_normal:
            kinds = [k | sg.LS_NORMAL for k in kinds]
        shifts = [ws[0].shifts[0]]
    else:
        ws = synth.batched_2d(args.batched_systems)
        kinds = [(sg.PATTERN_A if w.extra["pattern"] == "A" else sg.PATTERN_A2) | sg.PREC_FP32 for w in ws]
        if args.columns_normal:
            kinds = [k | sg.LS_NORMAL for k in kinds]
        shifts = [1.0] * len(ws)
    stream = torch.cuda.current_stream()
    ctx = sg.spai_ctx_create(stream.cuda_stream, 0)
    if args.columns_variant and args.columns_workload == "sweep3d":
        sg.spai_column_variant_set(args.columns_prec == "fp32", 25, 7, args.columns_variant)
    As, keep = [], []
    for w, sh in zip(ws, shifts):
        terms = [tuple(torch.as_tensor(np.ascontiguousarray(a), device="cuda") for a in t) for t in w.terms]
        aff = sg.spai_affine_create(ctx, [sg.csr(w.n, *t) for t in terms])
        _, nnz, rp, ci = sg.spai_affine_pattern(aff)
        va = torch.empty(nnz, dtype=torch.float64, device="cuda")
        sg.spai_assemble_shifted(ctx, aff, sh, w.params[0], w.alpha, w.beta, va)
        As.append(sg.csr(w.n, rp, ci, va, nnz))
        keep.append((aff, va, terms))

    def once():
        if args.columns_workload == "adaptive3d":
            sg.spai_pc_destroy(sg.spai_build_adaptive(ctx, As[0])[0])
            return
        if len(As) == 1:
            sg.spai_pc_destroy(sg.spai_build(ctx, As[0], kinds[0])[0])
            return
        for pc in sg.spai_build_batch(ctx, As, kinds)[0]:
            sg.spai_pc_destroy(pc)
    for _ in range(max(args.warmup, 1)):
        once()
    torch.cuda.synchronize()
    sg.spai_ctx_profile(ctx, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        once()
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) / max(args.steps, 1)
    prof = [sg.spai_ctx_profile_entry(ctx, i) for i in range(sg.spai_ctx_profile_count(ctx))]
    sg.spai_ctx_profile(ctx, 0)
    fp32_rate = max(sg.spai_measure_fp32_rate(ctx) for _ in range(3))
    for aff, _, _ in keep:
        sg.spai_affine_destroy(aff)
    sg.spai_ctx_destroy(ctx)
    col_unit = "fp32" if args.columns_prec == "fp32" else "fp64"
    roofs = {}
    for f in prof:
        if f["name"] == "spai_columns":
            r = roofline_entry(f, n=sum(w.n for w in ws), s=1, fp32_probe=fp32_rate, unit=col_unit)
            roofs[f["name"]] = {k: r[k] for k in ("bound", "achieved", "peak", "unit", "frac", "alu_frac",
                                                  "peak_source")}
    print(json.dumps({"kernel_case": "columns", "workload": args.columns_workload, "precision": args.columns_prec,
                      "fp32_tflops_measured": fp32_rate, "roofline": roofs,
                      "variant": args.columns_variant or "tuned",
                      "least_squares": "normal equations" if args.columns_normal else "Householder QR",
                      "systems": len(ws), "columns": sum(w.n for w in ws),
                      "steps": args.steps, "build_ms": 1e3 * wall,
                      "device_ms_per_build": {f["name"]: round(f["ms"] / max(args.steps, 1), 3) for f in prof}}),
          flush=True)


def run_spmm_case(args):
    """Y = A X on its own at the sweep's size: A(p_1, s_1) of the 3D side^3 7-point workload,
    X n x 8; `spmm32` the FP32 operator of the mixed solve, `spmm` the FP64 product."""
    import torch
    import paper_1809_06574_gb300 as sg
    import synth
    w = synth.grid3d_7pt(side=args.side, nparams=2)
    n, s = w.n, 8
    stream = torch.cuda.current_stream()
    ctx = sg.spai_ctx_create(stream.cuda_stream, 0)
    d_terms = [tuple(torch.as_tensor(np.ascontiguousarray(a), device="cuda") for a in tr) for tr in w.terms]
    aff = sg.spai_affine_create(ctx, [sg.csr(n, *tr) for tr in d_terms])
    _, nnz, rp, ci = sg.spai_affine_pattern(aff)
    va = torch.empty(nnz, dtype=torch.float64, device="cuda")
    sg.spai_assemble_shifted(ctx, aff, w.shifts[0], w.params[0], w.alpha, w.beta, va)
    A = sg.csr(n, rp, ci, va, nnz)
    g = torch.Generator(device="cpu").manual_seed(0)
    X = torch.randn(s, n, dtype=torch.float64, generator=g).cuda()
    Y = torch.empty_like(X)
    f = sg.spai_spmm_fp32 if args.kernel == "spmm32" else sg.spai_spmm
    for _ in range(max(args.warmup, 1)):
        f(ctx, A, s, X, n, Y, n)
    sg.spai_ctx_profile(ctx, 1)
    for _ in range(args.steps):
        f(ctx, A, s, X, n, Y, n)
    torch.cuda.synchronize()
    prof = [sg.spai_ctx_profile_entry(ctx, i) for i in range(sg.spai_ctx_profile_count(ctx))]
    prof = [p for p in prof if not p["name"].startswith("idle:")]
    sg.spai_affine_destroy(aff)
    sg.spai_ctx_destroy(ctx)
    fams = {p["name"]: roofline_entry(p, n=n, s=s) for p in prof}
    print(json.dumps({"kernel_case": args.kernel, "n": n, "nnz": nnz, "s": s, "steps": args.steps,
                      "families": fams}), flush=True)


def run_kernel_case(args):
    """One kernel on its own at the sweep's size: H = V^T W (dot) or W -= V H (update)."""
    import torch
    import paper_1809_06574_gb300 as sg
    if args.kernel == "columns":
        run_columns_case(args)
        return
    if args.kernel in ("spmm32", "spmm"):
        run_spmm_case(args)
        return
    n, s, nb = args.side ** 3, 8, args.nblk
    g = torch.Generator(device="cpu").manual_seed(0)
    # basis-like blocks: entries of unit-norm columns (the digit kernels take |v| < 2)
    V = (torch.randn(nb, n, s, dtype=torch.float64, generator=g) / n ** 0.5).cuda()
    W = torch.randn(n, s, dtype=torch.float64, generator=g).cuda()
    H = torch.randn(nb * s, s, dtype=torch.float64, generator=g).cuda()
    stream = torch.cuda.current_stream()
    ctx = sg.spai_ctx_create(stream.cuda_stream, 0)
    method = sg.ORTH_TENSOR if args.orth == "tensor" else sg.ORTH_FP64

    def once():
        if args.kernel == "dot":
            sg.spai_block_gram(ctx, s, n, nb, V, W, H, method)
        else:
            sg.spai_block_update(ctx, s, n, nb, V, H, W, -1.0, method)
    for _ in range(max(args.warmup, 1)):
        once()
    sg.spai_ctx_profile(ctx, 1)
    for _ in range(args.steps):
        once()
    torch.cuda.synchronize()
    prof = [sg.spai_ctx_profile_entry(ctx, i) for i in range(sg.spai_ctx_profile_count(ctx))]
    prof = [f for f in prof if not f["name"].startswith("idle:")]
    sg.spai_ctx_destroy(ctx)
    fams = {f["name"]: roofline_entry(f, n=n, s=s) for f in prof}
    print(json.dumps({"kernel_case": args.kernel, "n": n, "s": s, "nblk": nb, "orth": args.orth,
                      "steps": args.steps, "families": fams}), flush=True)


# ------------------------------------------------------------------------------ replicas
def aggregate_replicas(dist, torch, device, t_local, solves):
    """Whole-job figures of N independent replicas (one per rank, no data exchange):
    the slowest rank's time and the solves of all ranks.  dist None: one process."""
    if dist is None:
        return t_local, float(solves)
    t = torch.tensor([t_local, float(solves)], dtype=torch.float64, device=device)
    tm = t.clone()
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    ts = t.clone()
    dist.all_reduce(ts, op=dist.ReduceOp.SUM)
    return tm[0].item(), ts[1].item()


# ------------------------------------------------------------------------------- oracle
def oracle_sample(side, nparams, nsys, seed=0):
    """Time the CPU oracle on the first `nsys` systems of the sweep (build, then updates)."""
    import oracle
    import synth
    w = synth.grid3d_7pt(side=side, nparams=nparams, seed=seed)
    n = w.n
    s = w.shifts[0]
    t0 = time.perf_counter()
    base = None
    iters = []
    for i in range(nsys):
        p = w.params[i]
        A = oracle.assemble(w.terms, oracle.coefficients(p, s), n)
        if i == 0:
            base = oracle.spai_build(A, n)
            P = base
        else:
            P = oracle.spai_update(base, A, n)
        X, info = oracle.block_gmres(oracle.csr_apply(A, n), P.apply, w.B, w.restart, w.tol, 50)
        assert info["converged"]
        iters.append(info["iterations"])
    dt = time.perf_counter() - t0
    return nsys / dt, dt, iters


_ORACLE_W = {}


def _oracle_system(job):
    """One system of the sweep on the oracle, in a single-threaded worker process:
    assemble A(p, s), SPAI build, right-preconditioned block GMRES to the tolerance.
    Returns (seconds, iterations); the workload is generated once per process."""
    import oracle
    import synth
    side, nparams, si, pi = job
    key = (side, nparams)
    if key not in _ORACLE_W:
        _ORACLE_W[key] = synth.grid3d_7pt(side=side, nparams=nparams)
    w = _ORACLE_W[key]
    n = w.n
    t0 = time.perf_counter()
    A = oracle.assemble(w.terms, oracle.coefficients(w.params[pi], w.shifts[si]), n)
    P = oracle.spai_build(A, n)
    X, info = oracle.block_gmres(oracle.csr_apply(A, n), P.apply, w.B, w.restart, w.tol, 50)
    assert info["converged"]
    return time.perf_counter() - t0, info["iterations"]


class OraclePool:
    """One single-threaded oracle process per host core (spawned: no CUDA state is
    inherited), each solving whole systems of the sweep; `cores` is the number of processes,
    each with one BLAS / OpenMP thread."""

    def __init__(self, side, nparams):
        import multiprocessing as mp
        self.cores = os.cpu_count() or 1
        self.side, self.nparams = side, nparams
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(self.cores)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.round = 0

    def run_round(self):
        """Every process solves one system (shift k % 3, parameter (round + k) % nparams)."""
        jobs = [(self.side, self.nparams, k % 3, (self.round + k) % self.nparams) for k in range(self.cores)]
        self.round += 1
        t0 = time.perf_counter()
        out = self.pool.map(_oracle_system, jobs, chunksize=1)
        return time.perf_counter() - t0, out

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(side, nparams):
    """The oracle on all host cores: one warm-up round (each process generates the workload),
    then one timed round of one solve per process; solves / wall time of the round."""
    try:
        pool = OraclePool(side, nparams)
        pool.run_round()
        wall, out = pool.run_round()
        pool.close()
    except Exception as e:  # the baseline is reported, never required
        return {"value": None, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
                "sample": f"failed: {str(e)[-200:]}"}
    its = [o[1] for o in out]
    return {"value": len(out) / wall, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "sample": f"{len(out)} systems of the sweep at once (shifts and parameters spread over the "
                      f"processes), each assemble + SPAI build + block GMRES(50) to 1e-8 in its own "
                      f"single-threaded process, one per host core; {wall:.1f} s wall; GMRES iterations "
                      f"{min(its)}-{max(its)}; FP64 C (SPAI, sparse products) + numpy (block GMRES)"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import synth
    w = synth.grid3d_7pt(side=args.side, nparams=args.nparams)
    pool = OraclePool(args.side, args.nparams)
    pool.run_round()  # generates the workload in every process
    for _ in range(max(0, args.warmup - 1)):
        pool.run_round()
    total, solves = 0.0, 0
    for _ in range(args.steps):
        dt, out = pool.run_round()
        total += dt
        solves += len(out)
    pool.close()
    value = solves / total
    nnz = 7 * w.n - 6 * w.dims[0] ** 2
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(w, nnz),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                         "sample": f"each step: {pool.cores} systems of the sweep at once, one per "
                                   f"single-threaded oracle process (one per host core): assemble, SPAI "
                                   f"build, block GMRES(50) to 1e-8"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------- serving
def serve_trace(sg, torch, systems, Bs, trace, **opts):
    """Replay `trace` open-loop against a fresh server: each request is submitted at its
    arrival time (latency counts from that time, however late the submit), the solution
    is returned to host memory.  Returns the per-request results and the server stats."""
    srv = sg.spai_server_create(**opts)
    try:
        ids = [sg.spai_server_add_shifted_system(srv, [sg.csr(w.n, *t) for t in w.terms], w.alpha, w.beta) for w in systems]
        tickets = []
        done = []
        import queue as _q
        pending = _q.Queue()

        def collect():
            while True:
                item = pending.get()
                if item is None:
                    return
                tk, X = item
                done.append(sg.spai_server_wait(srv, tk))
                del X

        col = threading.Thread(target=collect, daemon=True)
        col.start()
        t0 = sg.spai_server_clock(srv) + 0.05
        for (ta, sy, p, s, nrhs) in trace:
            delay = t0 + ta - sg.spai_server_clock(srv)
            if delay > 0:
                time.sleep(delay)
            w = systems[sy]
            X = np.empty((w.n, nrhs), order="F")
            tk = sg.spai_server_submit(srv, ids[sy], nrhs, p, s, None, Bs[sy], X,
                                       t_arrival=t0 + ta)
            tickets.append(tk)
            pending.put((tk, X))
        pending.put(None)
        col.join()
        stats = sg.spai_server_stats_get(srv)
    finally:
        sg.spai_server_destroy(srv)
    return done, stats


def serving_summary(res, stats, n_of):
    lat = np.array([r["t_done"] - r["t_arrival"] for r in res])
    ok = [r for r in res if r["status"] == 0]
    span = max(r["t_done"] for r in res) - min(r["t_arrival"] for r in res)
    routes = {"build": 0, "update": 0, "reuse": 0}
    for r in res:
        routes[("build", "update", "reuse")[r["route"]]] += 1
    return {"requests": len(res), "completed_ok": len(ok), "value": len(ok) / span, "unit": UNIT,
            "span_s": round(span, 3),
            "latency_ms": {"p50": round(1e3 * float(np.percentile(lat, 50)), 2),
                           "p90": round(1e3 * float(np.percentile(lat, 90)), 2),
                           "p99": round(1e3 * float(np.percentile(lat, 99)), 2),
                           "max": round(1e3 * float(lat.max()), 2)},
            "routes": routes, "max_rel_residual": max(r["max_rel_residual"] for r in ok) if ok else None,
            "mem_peak_gb": round(stats["mem_peak"] / 1e9, 3), "evictions": stats["evictions"],
            "waits_for_memory": stats["waits_for_memory"]}


def run_serving(args, sg, torch):
    """Served (concurrent slots, cached builds routed to updates, FP32 factors) against FIFO
    plain FP64 (one slot, a SPAI build per request) on the same Poisson trace."""
    import synth
    systems = synth.serving_pool()
    Bs = [torch.from_numpy(np.asfortranarray(w.B).T.copy()).pin_memory() for w in systems]  # (8, n): column-major n x 8
    trace = synth.serving_trace(args.serve_rate, args.serve_seconds, len(systems))
    common = dict(restart=30, max_cycles=100, tol=1e-8)
    served = dict(slots=args.serve_slots, reuse=True, radius=0.05, pattern_kind=sg.PREC_FP32 | sg.LS_NORMAL,
                  mem_budget=40 << 30, precision=sg.SOLVE_MIXED, **common)
    # warm-up on a discarded server (module load, allocator pools); the timed server starts cold
    serve_trace(sg, torch, systems, Bs, [(0.0, i, 0.5, 1.0, 8) for i in range(len(systems))], **served)
    res, st = serve_trace(sg, torch, systems, Bs, trace, **served)
    out = serving_summary(res, st, None)
    fifo_trace = [r for r in trace if r[0] < args.serve_fifo_seconds]
    res_f, st_f = serve_trace(sg, torch, systems, Bs, fifo_trace, slots=1, reuse=False, mem_budget=40 << 30,
                              **common)
    fifo = serving_summary(res_f, st_f, None)
    # offered rates above the first: where does the server stop keeping up?
    rate_sweep = []
    for rate in [float(x) for x in args.serve_rates.split(",") if x]:
        tr = synth.serving_trace(rate, args.serve_rate_seconds, len(systems))
        r_, s_ = serve_trace(sg, torch, systems, Bs, tr, **served)
        sm = serving_summary(r_, s_, None)
        rate_sweep.append({"offered": rate, "requests": sm["requests"], "served": round(sm["value"], 1),
                           "p50_ms": sm["latency_ms"]["p50"], "p99_ms": sm["latency_ms"]["p99"],
                           "routes": sm["routes"]})
    nbar = float(np.mean([systems[sy].n for _, sy, _, _, _ in trace]))
    return {
        "workload": f"Poisson {args.serve_rate:g} req/s for {args.serve_seconds:g} s over 16 3D 7-point grids "
                    f"(sides {synth.SERVE_SIDES[0]}-{synth.SERVE_SIDES[-1]}, mean n of the requests {nbar:.0f}); 70 % within "
                    f"0.05 of a served p; s in {{0.5,1,2}}; nrhs in {{1,4,8}}; block GMRES(30) to 1e-8; "
                    f"40 GB budget; solutions returned to host memory",
        "served": {**out, "slots": args.serve_slots, "factors": "f32", "solve": "mixed (f32 operator, f64 refinement)",
                   "reuse_radius": 0.05},
        "rate_sweep": rate_sweep,
        "fifo_plain_fp64": {**fifo, "slots": 1, "factors": "f64", "reuse": False,
                            "trace": f"the first {args.serve_fifo_seconds:g} s of the same arrivals"},
        "served_over_fifo": out["value"] / fifo["value"] if fifo["value"] else None,
    }


def run_served_sweep(args, sg, torch, w, steps, warmup=1):
    """The headline sweep's systems (every p at every s, 8 right-hand sides) submitted to the
    server all at once, a closed loop at saturation: served capacity = solves / makespan
    (first submit to last completion, device-resident B and X).  The server runs the served
    form -- FP32 factors, the FP32 operator with FP64 refinement, one build per shift cached
    and every other parameter routed to an update from it (radius covering the sweep's p
    range, as the plain sweep's one build per shift) -- on `slots` = bench workers."""
    dev = torch.device("cuda", torch.cuda.current_device())
    n = w.n
    d_terms = [tuple(torch.as_tensor(np.ascontiguousarray(a), device=dev) for a in t) for t in w.terms]
    B = torch.as_tensor(np.ascontiguousarray(w.B.T), device=dev)  # (8, n): column-major n x 8
    reqs = [(p, s) for s in w.shifts for p in w.params]
    Xs = [torch.empty((int(w.B.shape[1]), n), dtype=torch.float64, device=dev) for _ in reqs]
    opts = dict(slots=args.workers, reuse=True, radius=1.0, pattern_kind=sg.PATTERN_A | sg.PREC_FP32 | sg.LS_NORMAL,
                restart=w.restart, max_cycles=50, tol=w.tol, precision=sg.SOLVE_MIXED)
    spans, lats, iters, routes = [], [], [], {"build": 0, "update": 0, "reuse": 0}
    for it in range(warmup + steps):
        srv = sg.spai_server_create(**opts)
        try:
            sid = sg.spai_server_add_shifted_system(srv, [sg.csr(n, *t) for t in d_terms], w.alpha, w.beta)
            torch.cuda.synchronize()
            t0 = sg.spai_server_clock(srv)
            tickets = [sg.spai_server_submit(srv, sid, int(w.B.shape[1]), p, s, None, B, X, t_arrival=t0)
                       for (p, s), X in zip(reqs, Xs)]
            res = [sg.spai_server_wait(srv, tk) for tk in tickets]
        finally:
            sg.spai_server_destroy(srv)
        bad = [r for r in res if r["status"] != 0]
        if bad:
            raise RuntimeError(f"served sweep: {len(bad)} requests failed: {bad[0]}")
        if it < warmup:
            continue
        spans.append(max(r["t_done"] for r in res) - t0)
        lats.extend(r["t_done"] - r["t_arrival"] for r in res)
        iters.extend(r["iterations"] for r in res)
        for r in res:
            routes[("build", "update", "reuse")[r["route"]]] += 1
    lat = np.array(lats)
    return {"value": len(reqs) * steps / sum(spans), "unit": UNIT, "steps": steps,
            "ms_per_step": 1e3 * sum(spans) / steps,
            "latency_ms": {"p50": round(1e3 * float(np.percentile(lat, 50)), 2),
                           "p99": round(1e3 * float(np.percentile(lat, 99)), 2)},
            "gmres_iterations_mean": float(np.mean(iters)), "routes": routes, "slots": args.workers,
            "form": "server, FP32 factors (normal equations), FP32 operator + FP64 refinement, one cached build per shift "
                    "and updates from it, all 60 requests at once (closed loop)"}


# ------------------------------------------------------------------------------- batched
def run_batched(args, sg, torch):
    """256 independent 2D 5-point systems (grid sides ~ U{48..256}, each with its own seed,
    p ~ U[0.1, 1], s = 1), SPAI pattern of A for half of them and of A^2 for the other half,
    FP32 factors: all SPAI builds in one spai_build_batch call (one persistent launch per
    tile shape), then every system solved (4 RHS, block GMRES(30) to 1e-8 in FP64) in one
    block_solve_batch call (in lockstep, each system leaving it when its residual estimate
    meets tol).  Beside them: the same builds one
    spai_build call at a time, and the same solves one block_solve per system on
    `batched_workers` streams."""
    import synth
    from concurrent.futures import ThreadPoolExecutor
    nsys = args.batched_systems
    ws = synth.batched_2d(nsys)
    kinds = [(sg.PATTERN_A if w.extra["pattern"] == "A" else sg.PATTERN_A2) | sg.PREC_FP32 for w in ws]
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    ctx = sg.spai_ctx_create(stream.cuda_stream, 0)
    systems = []
    for w in ws:
        aff = sg.spai_affine_create(ctx, [sg.csr(w.n, *t) for t in w.terms])
        _, nnz, rp, ci = sg.spai_affine_pattern(aff)
        va = torch.empty(nnz, dtype=torch.float64, device=dev)
        sg.spai_assemble_shifted(ctx, aff, 1.0, w.params[0], w.alpha, w.beta, va)
        B = torch.as_tensor(np.ascontiguousarray(w.B.T), device=dev)
        systems.append({"w": w, "aff": aff, "va": va, "A": sg.csr(w.n, rp, ci, va, nnz), "B": B})
    As = [y["A"] for y in systems]
    # tune the tile shapes once (a small batch with both shapes), as a long-running process would
    for pc in sg.spai_build_batch(ctx, As[:2], kinds[:2])[0]:
        sg.spai_pc_destroy(pc)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pcs, _ = sg.spai_build_batch(ctx, As, kinds)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    t0 = time.perf_counter()
    for A, k in zip(As, kinds):
        sg.spai_pc_destroy(sg.spai_build(ctx, A, k)[0])
    torch.cuda.synchronize()
    t_loop = time.perf_counter() - t0

    workers = [(torch.cuda.Stream(device=dev),) for _ in range(args.batched_workers)]
    wctx = [sg.spai_ctx_create(st.cuda_stream, 0) for (st,) in workers]
    Xs = [torch.zeros((4, y["w"].n), dtype=torch.float64, device=dev) for y in systems]
    iters = [0] * nsys

    def solve_share(k):
        for i in range(k, nsys, len(workers)):
            y = systems[i]
            n = y["w"].n
            with torch.cuda.stream(workers[k][0]):
                Xs[i].zero_()
            st, info, rel = sg.block_solve(wctx[k], y["A"], pcs[i], 4, y["B"], n, Xs[i], n, 30, 1e-8, 100)
            if not info["converged"]:
                raise RuntimeError(f"batched system {i} did not converge: {info}")
            iters[i] = info["iterations"]

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=len(workers)) as ex:
        list(ex.map(solve_share, range(len(workers))))
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t0
    # the same solves in lockstep: one block_solve_batch call over all systems, each leaving
    # the lockstep when it has converged
    for X in Xs:
        X.zero_()
    Bs = [y["B"] for y in systems]
    sg.block_solve_batch(ctx, As[:2], pcs[:2], 4, Bs[:2], Xs[:2], 30, 1e-8, 100)  # warm-up
    for X in Xs:
        X.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, infos = sg.block_solve_batch(ctx, As, pcs, 4, Bs, Xs, 30, 1e-8, 100)
    torch.cuda.synchronize()
    t_solve_b = time.perf_counter() - t0
    if not all(i["converged"] for i in infos):
        raise RuntimeError("batched solve did not converge")
    for c in wctx:
        sg.spai_ctx_destroy(c)
    for pc in pcs:
        sg.spai_pc_destroy(pc)
    for y in systems:
        sg.spai_affine_destroy(y["aff"])
    sg.spai_ctx_destroy(ctx)
    ncols = int(sum(y["w"].n for y in systems))
    return {
        "workload": f"{nsys} independent 2D 5-point systems, sides U{{48..256}} (n {min(y['w'].n for y in systems)}-"
                    f"{max(y['w'].n for y in systems)}, {ncols} columns in all), p ~ U[0.1,1], s=1, SPAI pattern of A "
                    f"(half) / A^2 (half), FP32 factors, 4 RHS, block GMRES(30) to 1e-8 in FP64",
        "build_batch_ms": 1e3 * t_batch, "build_one_by_one_ms": 1e3 * t_loop, "batch_speedup": t_loop / t_batch,
        "solve_batch_ms": 1e3 * t_solve_b, "solve_streams_ms": 1e3 * t_solve, "workers": len(workers),
        "value": nsys / (t_batch + t_solve_b), "unit": UNIT,
        "value_streams": nsys / (t_batch + t_solve),
        "gmres_iterations": {"mean": float(np.mean(iters)), "max": int(max(iters)),
                             "batch_mean": float(np.mean([i["iterations"] for i in infos])),
                             "batch_max": int(max(i["iterations"] for i in infos))},
        "max_rel_residual": max(i["max_rel_residual"] for i in infos),
    }


# --------------------------------------------------------------------- block vs single RHS
def run_block_vs_single(sg, torch, ctx, w, nsys=5):
    """Block GMRES(m) with all 8 right-hand sides at once against 8 single-RHS GMRES(m)
    solves of the same systems (Sec. 2.1: block methods share one Krylov space), on the
    first `nsys` parameters of the shift s = 1 (SPAI build at the first, updates after),
    one stream, FP64 throughout."""
    nsys = min(nsys, len(w.params))  # a sweep reduced by --nparams has fewer parameters
    n, nr = w.n, int(w.B.shape[1])
    dev = torch.device("cuda", torch.cuda.current_device())
    d_terms = [tuple(torch.as_tensor(np.ascontiguousarray(a), device=dev) for a in t) for t in w.terms]
    aff = sg.spai_affine_create(ctx, [sg.csr(n, *t) for t in d_terms])
    _, nnz, rp, ci = sg.spai_affine_pattern(aff)
    vals = [torch.empty(nnz, dtype=torch.float64, device=dev) for _ in range(nsys)]
    As, pcs = [], []
    for i in range(nsys):
        sg.spai_assemble_shifted(ctx, aff, 1.0, w.params[i], w.alpha, w.beta, vals[i])
        As.append(sg.csr(n, rp, ci, vals[i], nnz))
        pcs.append(sg.spai_build(ctx, As[0])[0] if i == 0 else sg.spai_update(ctx, pcs[0], As[i])[0])
    B = torch.as_tensor(np.ascontiguousarray(w.B.T), device=dev)  # (8, n): column c at row c
    X = torch.zeros((nr, n), dtype=torch.float64, device=dev)

    def block():
        its = 0
        for A, pc in zip(As, pcs):
            X.zero_()
            its += sg.block_solve(ctx, A, pc, nr, B, n, X, n, w.restart, w.tol, 50)[1]["iterations"]
        return its

    def single():
        its = 0
        for A, pc in zip(As, pcs):
            X.zero_()
            for c in range(nr):
                its += sg.block_solve(ctx, A, pc, 1, B[c], n, X[c], n, w.restart, w.tol, 200)[1]["iterations"]
        return its

    out = {}
    for name, f in (("block", block), ("single", single)):
        f()  # warm-up (workspace sizes)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its = f()
        torch.cuda.synchronize()
        out[name] = {"ms_per_system": 1e3 * (time.perf_counter() - t0) / nsys, "iterations_per_system": its / nsys}
    for i in range(nsys - 1, -1, -1):
        sg.spai_pc_destroy(pcs[i])
    sg.spai_affine_destroy(aff)
    return {"systems": nsys, "shift": 1.0, **out,
            "block_saving": 1.0 - out["block"]["ms_per_system"] / out["single"]["ms_per_system"],
            "note": "one stream; block = one s = 8 solve per system, single = eight s = 1 solves; "
                    "iterations are Arnoldi steps (block steps for the block solve)"}


def run_update_order(sg, torch, ctx, w, nparams=4):
    """The two update orders of Sec. 2.4 on the same systems (the first `nparams` parameters
    x the three shifts), one stream, FP64: over p -- per shift, SPAI built at the first
    parameter, Q_l updates for the others (the sweep's order) -- and over s -- per
    parameter, SPAI built at the first shift, updates for the other shifts
    (min ||A(s_1, p) - A(s_k, p) Q||_F, P = Q P_1).  Each system is then solved (block
    GMRES(m), 8 RHS); reported: time per solve including builds and updates, and the mean
    iteration count of each order."""
    n, nr = w.n, int(w.B.shape[1])
    dev = torch.device("cuda", torch.cuda.current_device())
    d_terms = [tuple(torch.as_tensor(np.ascontiguousarray(a), device=dev) for a in t) for t in w.terms]
    aff = sg.spai_affine_create(ctx, [sg.csr(n, *t) for t in d_terms])
    _, nnz, rp, ci = sg.spai_affine_pattern(aff)
    ps, ss = list(w.params[:nparams]), list(w.shifts)
    vals = {}
    for p in ps:
        for sh in ss:
            v = torch.empty(nnz, dtype=torch.float64, device=dev)
            sg.spai_assemble_shifted(ctx, aff, sh, p, w.alpha, w.beta, v)
            vals[(p, sh)] = sg.csr(n, rp, ci, v, nnz)
    B = torch.as_tensor(np.ascontiguousarray(w.B.T), device=dev)
    X = torch.zeros((nr, n), dtype=torch.float64, device=dev)

    def run(groups):
        """groups: lists of (p, s) keys; the first of a group is built, the rest updated."""
        its = []
        for g in groups:
            base = sg.spai_build(ctx, vals[g[0]])[0]
            for key in g:
                pc = base if key == g[0] else sg.spai_update(ctx, base, vals[key])[0]
                X.zero_()
                info = sg.block_solve(ctx, vals[key], pc, nr, B, n, X, n, w.restart, w.tol, 50)[1]
                assert info["converged"], info
                its.append(info["iterations"])
                if pc is not base:
                    sg.spai_pc_destroy(pc)
            sg.spai_pc_destroy(base)
        return its

    orders = {"over_p": [[(p, sh) for p in ps] for sh in ss], "over_s": [[(p, sh) for sh in ss] for p in ps]}
    out = {}
    for name, groups in orders.items():
        run(groups)  # warm-up (workspaces, kernel choices)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its = run(groups)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[name] = {"builds": len(groups), "updates": len(its) - len(groups), "ms_per_solve": 1e3 * dt / len(its),
                     "gmres_iterations_mean": float(np.mean(its)), "gmres_iterations_max": int(max(its))}
    sg.spai_affine_destroy(aff)
    return {"systems": len(ps) * len(ss), "params": ps, "shifts": ss, **out,
            "note": "one stream, FP64; over_p = one SPAI per shift updated across p (the sweep's order), "
                    "over_s = one SPAI per parameter updated across s"}


def run_adaptive(sg, torch, ctx, w, nparams=3):
    """Adaptive SPAI (pattern grown per column to the paper's MSPAI tolerance 1e-4, at most
    5 steps of 5 columns) on the sweep's matrices at the first shift: built at p_1, then
    for the next `nparams` parameters an update from it (the base's pattern: no search,
    Sec. 2.3-2.4) against a rebuild with its own search, each followed by the block GMRES
    solve (8 RHS).  One stream, FP64; the paper's comparison (SPAI vs SPAI update, Sec. 3)."""
    n, nr = w.n, int(w.B.shape[1])
    dev = torch.device("cuda", torch.cuda.current_device())
    d_terms = [tuple(torch.as_tensor(np.ascontiguousarray(a), device=dev) for a in t) for t in w.terms]
    aff = sg.spai_affine_create(ctx, [sg.csr(n, *t) for t in d_terms])
    _, nnz, rp, ci = sg.spai_affine_pattern(aff)
    sh = w.shifts[0]
    vals = [torch.empty(nnz, dtype=torch.float64, device=dev) for _ in range(nparams + 1)]
    As = []
    for i, v in enumerate(vals):
        sg.spai_assemble_shifted(ctx, aff, sh, w.params[i], w.alpha, w.beta, v)
        As.append(sg.csr(n, rp, ci, v, nnz))
    B = torch.as_tensor(np.ascontiguousarray(w.B.T), device=dev)
    X = torch.zeros((nr, n), dtype=torch.float64, device=dev)

    def timed(f):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = f()
        torch.cuda.synchronize()
        return r, 1e3 * (time.perf_counter() - t0)

    def solve(A, pc):
        X.zero_()
        info = sg.block_solve(ctx, A, pc, nr, B, n, X, n, w.restart, w.tol, 50)[1]
        assert info["converged"], info
        return info["iterations"]

    sg.spai_pc_destroy(sg.spai_build_adaptive(ctx, As[0])[0])  # warm-up (kernel choices, pools)
    base, t_base = timed(lambda: sg.spai_build_adaptive(ctx, As[0])[0])
    nnz_p = sg.spai_pc_info(base)["nnz"]
    rows = []
    for i in range(1, nparams + 1):
        q, t_upd = timed(lambda: sg.spai_update(ctx, base, As[i])[0])
        it_upd, t_su = timed(lambda: solve(As[i], q))
        sg.spai_pc_destroy(q)
        pc, t_reb = timed(lambda: sg.spai_build_adaptive(ctx, As[i])[0])
        it_reb, t_sr = timed(lambda: solve(As[i], pc))
        sg.spai_pc_destroy(pc)
        fixed = sg.spai_build(ctx, As[i], sg.PATTERN_A)[0]
        it_fix = solve(As[i], fixed)
        sg.spai_pc_destroy(fixed)
        rows.append({"p": w.params[i], "update_ms": t_upd, "rebuild_ms": t_reb, "solve_after_update_ms": t_su,
                     "solve_after_rebuild_ms": t_sr, "iterations_update": it_upd, "iterations_rebuild": it_reb,
                     "iterations_fixed_pattern_A": it_fix})
    sg.spai_pc_destroy(base)
    sg.spai_affine_destroy(aff)
    upd = float(np.mean([r["update_ms"] for r in rows]))
    reb = float(np.mean([r["rebuild_ms"] for r in rows]))
    tot_u = float(np.mean([r["update_ms"] + r["solve_after_update_ms"] for r in rows]))
    tot_r = float(np.mean([r["rebuild_ms"] + r["solve_after_rebuild_ms"] for r in rows]))
    return {"workload": f"3d-64^3-7pt at s={sh}: adaptive SPAI (eps 1e-4, 5 steps x 5 columns) at p_1, "
                        f"update vs rebuild at {nparams} further p, block GMRES({w.restart}) 8 RHS, FP64",
            "build_ms": t_base, "nnz_per_column": nnz_p / n, "update_ms": upd, "rebuild_ms": reb,
            "update_saving": 1.0 - upd / reb, "update_plus_solve_ms": tot_u, "rebuild_plus_solve_ms": tot_r,
            "update_plus_solve_saving": 1.0 - tot_u / tot_r, "per_parameter": rows}


# ------------------------------------------------------------------------------- large
def run_large(args, sg, torch):
    """3D side^3 27-point workload (side 128: n = 2,097,152, 27 nnz per column, 16 RHS):
    SPAI in FP32 stored as BF16 at the first p, then for a sample of the other p an update
    (Table 1, first approach) + block GMRES(30) solve, against a rebuild + solve at the
    same p; the FP64 build is timed once beside them."""
    import synth
    w = synth.grid3d_27pt(side=args.large_side, nparams=50)
    n, s = w.n, int(w.B.shape[1])
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    ctx = sg.spai_ctx_create(stream.cuda_stream, 0)
    d_terms = [tuple(torch.as_tensor(np.ascontiguousarray(a), device=dev) for a in t) for t in w.terms]
    aff = sg.spai_affine_create(ctx, [sg.csr(n, *t) for t in d_terms])
    _, nnz, rp, ci = sg.spai_affine_pattern(aff)
    va = [torch.empty(nnz, dtype=torch.float64, device=dev) for _ in range(2)]
    B = torch.as_tensor(np.ascontiguousarray(w.B.T), device=dev)
    X = torch.zeros((s, n), dtype=torch.float64, device=dev)

    def timed(f):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = f()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t0

    def solve(A, pc, precision=sg.SOLVE_MIXED):
        # the workload's solve: FP32 SpMM (the FP32 operator) with FP64 refinement to 1e-8
        X.zero_()
        st, info, rel = sg.block_solve(ctx, A, pc, s, B, n, X, n, 30, 1e-8, 100, precision=precision)
        assert info["converged"], info
        return info

    # the library tunes its column kernel once per tile shape and process; a long-running
    # process has done so before it builds at this size: tune the FP64 shape (|I| <= 125,
    # |J| <= 27) on a small grid of the same stencil first
    ws = synth.grid3d_27pt(side=24, nparams=2)
    sm_terms = [tuple(torch.as_tensor(np.ascontiguousarray(a), device=dev) for a in t) for t in ws.terms]
    sm_aff = sg.spai_affine_create(ctx, [sg.csr(ws.n, *t) for t in sm_terms])
    _, sm_nnz, sm_rp, sm_ci = sg.spai_affine_pattern(sm_aff)
    sm_va = torch.empty(sm_nnz, dtype=torch.float64, device=dev)
    sg.spai_assemble_shifted(ctx, sm_aff, 1.0, ws.params[0], ws.alpha, ws.beta, sm_va)
    sg.spai_pc_destroy(sg.spai_build(ctx, sg.csr(ws.n, sm_rp, sm_ci, sm_va, sm_nnz), sg.PATTERN_A)[0])
    sg.spai_affine_destroy(sm_aff)
    sg.spai_assemble_shifted(ctx, aff, 1.0, w.params[0], w.alpha, w.beta, va[0])
    A1 = sg.csr(n, rp, ci, va[0], nnz)
    pc64, t_b64 = timed(lambda: sg.spai_build(ctx, A1, sg.PATTERN_A)[0])
    sg.spai_pc_destroy(pc64)
    sg.spai_pc_destroy(sg.spai_build(ctx, A1, sg.PATTERN_A | sg.PREC_BF16)[0])  # warm-up
    base, t_b16 = timed(lambda: sg.spai_build(ctx, A1, sg.PATTERN_A | sg.PREC_BF16)[0])
    solve(A1, base)  # warm-up of the solve path at this size
    rows = []
    for p in w.params[1:1 + args.large_params]:
        sg.spai_assemble_shifted(ctx, aff, 1.0, p, w.alpha, w.beta, va[1])
        A = sg.csr(n, rp, ci, va[1], nnz)
        upd, t_u = timed(lambda: sg.spai_update(ctx, base, A, sg.UPDATE_FIRST | sg.PREC_BF16)[0])
        iu, t_su = timed(lambda: solve(A, upd))
        sg.spai_pc_destroy(upd)
        dgu, t_d = timed(lambda: sg.spai_update(ctx, base, A, sg.UPDATE_FIRST | sg.UPDATE_DIAGONAL |
                                                sg.PREC_BF16)[0])
        idg, t_sd = timed(lambda: solve(A, dgu))
        sg.spai_pc_destroy(dgu)
        reb, t_r = timed(lambda: sg.spai_build(ctx, A, sg.PATTERN_A | sg.PREC_BF16)[0])
        ir, t_sr = timed(lambda: solve(A, reb))
        if not rows:  # the same solve with FP64 products, once, for comparison
            i64, t_s64 = timed(lambda: solve(A, reb, sg.SOLVE_FP64))
        sg.spai_pc_destroy(reb)
        rows.append({"p": round(p, 4), "update_ms": 1e3 * t_u, "solve_after_update_ms": 1e3 * t_su,
                     "iterations_update": iu["iterations"],
                     "diagonal_update_ms": 1e3 * t_d, "solve_after_diagonal_update_ms": 1e3 * t_sd,
                     "iterations_diagonal_update": idg["iterations"], "rebuild_ms": 1e3 * t_r,
                     "solve_after_rebuild_ms": 1e3 * t_sr, "iterations_rebuild": ir["iterations"],
                     "max_rel_residual": max(iu["max_rel_residual"], idg["max_rel_residual"],
                                             ir["max_rel_residual"])})
    sg.spai_pc_destroy(base)
    sg.spai_affine_destroy(aff)
    sg.spai_ctx_destroy(ctx)
    upd_s = sum(r["update_ms"] + r["solve_after_update_ms"] for r in rows) / 1e3
    dg_s = sum(r["diagonal_update_ms"] + r["solve_after_diagonal_update_ms"] for r in rows) / 1e3
    reb_s = sum(r["rebuild_ms"] + r["solve_after_rebuild_ms"] for r in rows) / 1e3
    return {
        "workload": f"3d-{args.large_side}^3-27pt, n={n}, nnz={nnz}, {s} RHS, SPAI(pattern A) FP32 stored "
                    f"as BF16, block GMRES(30) with the FP32 operator and FP64 refinement to true residual "
                    f"1e-8; {len(rows)} of the 49 further p",
        "build_fp64_ms": 1e3 * t_b64, "build_bf16_ms": 1e3 * t_b16, "per_parameter": rows,
        "solve_after_rebuild_fp64_products_ms": 1e3 * t_s64, "iterations_fp64_products": i64["iterations"],
        "update_path_solves_per_s": len(rows) / upd_s, "rebuild_path_solves_per_s": len(rows) / reb_s,
        "update_saving": 1.0 - upd_s / reb_s,
        "diagonal_update_path_solves_per_s": len(rows) / dg_s, "diagonal_update_saving": 1.0 - dg_s / reb_s,
    }


# ------------------------------------------------------------------------------- GPU sweep
class Worker:
    """One host thread's share of the sweep: its own stream, context and buffers."""

    def __init__(self, sg, torch, n, s, nnz, dev, host_inputs):
        self.stream = torch.cuda.Stream(device=dev)
        self.ctx = sg.spai_ctx_create(self.stream.cuda_stream, 0)
        with torch.cuda.stream(self.stream):
            self.va = torch.empty(nnz, dtype=torch.float64, device=dev)
            if host_inputs:
                self.X = torch.zeros((s, n), dtype=torch.float64).pin_memory()
            else:
                self.X = torch.zeros((s, n), dtype=torch.float64, device=dev)
        self.rcs = {}  # block GCRO: a recycle space per shift


class Sweep:
    """One step = the whole parameter sweep: for every shift s a SPAI build at the first p,
    then (Table 1, first approach) an update per further p, and a block GMRES solve of
    every system.  The 60 systems are independent once their shift's base is built;
    `workers` host threads, each with its own stream and context, take them round-robin
    while the main context builds the bases."""

    def __init__(self, sg, torch, ctx, w, host_inputs=False, workers=1, prec=0, warm=False, solve_precision=0,
                 gcro_kmax=0):
        self.sg, self.torch, self.ctx, self.w = sg, torch, ctx, w
        self.prec = prec  # 0: FP64 factors; sg.PREC_FP32: FP32 least squares and factors
        self.solve_precision = solve_precision  # sg.SOLVE_MIXED: FP32 operator, FP64 refinement
        # gcro_kmax > 0: block GCRO, each worker carrying a recycle space of that many columns
        # per shift along its parameters (the span of its latest solutions of the shift)
        self.gcro_kmax = gcro_kmax
        # warm: a worker starts each solve from its previous solution of the same shift (all
        # systems share B, and neighbouring parameters have close solutions)
        self.warm = warm
        n = w.n
        self.n = n
        self.s = w.B.shape[1]
        dev = torch.device("cuda", torch.cuda.current_device())
        self.dev = dev
        self.host_inputs = host_inputs
        if host_inputs:
            # pinned host copies of the inputs; copied to the device inside every step
            self.h_terms = []
            for t in w.terms:
                self.h_terms.append(tuple(torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                                          for a in t))
            self.B = torch.from_numpy(np.ascontiguousarray(w.B.T)).pin_memory()
            self.aff = None
        else:
            self.d_terms = [tuple(torch.as_tensor(np.ascontiguousarray(a), device=dev) for a in t)
                            for t in w.terms]
            self.aff = sg.spai_affine_create(ctx, [sg.csr(n, *t) for t in self.d_terms])
            self.B = torch.as_tensor(np.ascontiguousarray(w.B.T), device=dev)
        nnz = sum(len(t[1]) for t in w.terms)  # upper bound of the union pattern
        self.vb = [torch.empty(nnz, dtype=torch.float64, device=dev) for _ in w.shifts]  # A(p_1, s) per shift
        self.workers = [Worker(sg, torch, n, self.s, nnz, dev, host_inputs) for _ in range(workers)]
        self.pool = None
        if workers > 1:
            from concurrent.futures import ThreadPoolExecutor
            self.pool = ThreadPoolExecutor(max_workers=workers)
        self.solves = 0
        self.iters = []
        self.cycles = []
        self.errors = []

    def close(self):
        if self.pool is not None:
            self.pool.shutdown()
        for wk in self.workers:
            for rc in wk.rcs.values():
                self.sg.spai_recycle_destroy(rc)
            self.sg.spai_ctx_destroy(wk.ctx)

    def h2d_bytes(self):
        tb = sum(a.numel() * a.element_size() for t in self.h_terms for a in t)
        nsys = len(self.w.params) * len(self.w.shifts)
        per = self.n * self.s * 8
        return tb + nsys * 2 * per  # terms once + B and the initial guess X0 per solve

    def d2h_bytes(self):
        return len(self.w.params) * len(self.w.shifts) * self.n * self.s * 8

    def _solve(self, wk, k, tasks, bases, A0s, ready, rp, ci, nnz):
        """Tasks k, k + W, ... of the flattened sweep on worker wk.  Task (si, i) is parameter
        i of shift si: it waits for that shift's base build; i == 0 solves with the base
        itself, the others assemble A(p_i, s), update the base (Table 1, first approach)
        and solve."""
        sg, torch, w, n = self.sg, self.torch, self.w, self.n
        out = []
        prev_si = -1
        for t in range(k, len(tasks), len(self.workers)):
            si, i = tasks[t]
            s = w.shifts[si]
            ready[si].wait()
            base = bases[si]
            if base is None:
                raise RuntimeError(f"the base build of shift {s} failed")
            if i == 0:
                A, pc = A0s[si], base
            else:
                sg.spai_assemble_shifted(wk.ctx, self.aff_now, s, w.params[i], w.alpha, w.beta, wk.va)
                A = sg.csr(n, rp, ci, wk.va, nnz)
                pc, _ = sg.spai_update(wk.ctx, base, A, sg.UPDATE_FIRST | self.prec)
            if not (self.warm and si == prev_si):
                with torch.cuda.stream(wk.stream):
                    wk.X.zero_()
            prev_si = si
            if self.gcro_kmax:
                if si not in wk.rcs:
                    wk.rcs[si] = sg.spai_recycle_create(wk.ctx, n, self.s, self.gcro_kmax)
                with torch.cuda.stream(wk.stream):
                    wk.X.zero_()
                st, info, rel = sg.block_solve_gcro(wk.ctx, A, pc, self.s, self.B, n, wk.X, n, w.restart, w.tol, 50,
                                                    wk.rcs[si], precision=self.solve_precision)
            else:
                st, info, rel = sg.block_solve(wk.ctx, A, pc, self.s, self.B, n, wk.X, n,
                                               w.restart, w.tol, 50, precision=self.solve_precision)
            if i > 0:
                sg.spai_pc_destroy(pc)
            if not info["converged"]:
                raise RuntimeError(f"solve did not converge: p={w.params[i]} s={s} {info}")
            out.append(info["iterations"])
            self.cycles.append(info["cycles"])
        return out

    def step(self):
        """The shifts' base builds run on the main context while the workers already solve:
        a worker reaching a shift whose base is not built yet waits for it, so the builds
        overlap the other shifts' solves and no shift waits for the last solve of the one
        before."""
        sg, torch, ctx, w, n = self.sg, self.torch, self.ctx, self.w, self.n
        aff = self.aff
        for wk in self.workers:  # every step starts without recycled spaces
            for rc in wk.rcs.values():
                sg.spai_recycle_clear(rc)
        if self.host_inputs:
            aff = sg.spai_affine_create(ctx, [sg.csr(n, *t) for t in self.h_terms])
        self.aff_now = aff
        _, nnz, rp, ci = sg.spai_affine_pattern(aff)
        tasks = [(si, i) for si in range(len(w.shifts)) for i in range(len(w.params))]
        bases = [None] * len(w.shifts)
        A0s = [None] * len(w.shifts)
        ready = [threading.Event() for _ in w.shifts]
        futs = []
        if self.pool is not None:
            futs = [self.pool.submit(self._solve, wk, k, tasks, bases, A0s, ready, rp, ci, nnz)
                    for k, wk in enumerate(self.workers)]
        try:
            for si, s in enumerate(w.shifts):
                sg.spai_assemble_shifted(ctx, aff, s, w.params[0], w.alpha, w.beta, self.vb[si])
                A0s[si] = sg.csr(n, rp, ci, self.vb[si], nnz)
                # returns with the build complete: its handle is then read-only for the workers
                bases[si] = sg.spai_build(ctx, A0s[si], sg.PATTERN_A | self.prec)[0]
                ready[si].set()
        finally:
            for e in ready:  # a failed build must not leave a worker waiting
                e.set()
        if self.pool is None:
            res = [self._solve(self.workers[0], 0, tasks, bases, A0s, ready, rp, ci, nnz)]
        else:
            res = [f.result() for f in futs]
        for r in res:
            self.solves += len(r)
            self.iters.extend(r)
        for b in bases:
            if b is not None:
                sg.spai_pc_destroy(b)
        if self.host_inputs:
            sg.spai_affine_destroy(aff)

    def profile(self, enable):
        for c in [self.ctx] + [wk.ctx for wk in self.workers]:
            self.sg.spai_ctx_profile(c, enable)

    def profile_entries(self):
        """Per-family totals summed over the step's contexts.  Idle families ("idle:...")
        are kept for the workers' streams only, averaged over the workers (the main
        context's stream waits between shifts by design)."""
        fam = {}
        nw = len(self.workers)
        for c in [self.ctx] + [wk.ctx for wk in self.workers]:
            for i in range(self.sg.spai_ctx_profile_count(c)):
                e = self.sg.spai_ctx_profile_entry(c, i)
                idle = e["name"].startswith("idle:")
                if idle and c == self.ctx:
                    continue
                f = fam.setdefault(e["name"], {"name": e["name"], "launches": 0, "ms": 0.0, "flops": 0.0,
                                               "bytes": 0.0})
                for k in ("launches", "ms", "flops", "bytes"):
                    f[k] += e[k] / (nw if idle else 1)
        return list(fam.values())


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.kernel:
        if rank == 0:
            run_kernel_case(args)
        return

    import synth
    w = synth.grid3d_7pt(side=args.side, nparams=args.nparams, seed=rank)
    nnz_expected = 7 * w.n - 6 * w.dims[0] ** 2

    # CPU baseline first, before any CUDA work in this process
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.side, args.nparams)

    import torch
    import paper_1809_06574_gb300 as sg
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    if args.serve_only:
        if rank == 0:
            print(json.dumps({"serving": run_serving(args, sg, torch)}), flush=True)
        return
    if args.large_only:
        if rank == 0:
            print(json.dumps({"large": run_large(args, sg, torch)}), flush=True)
        return
    if args.batched_only:
        if rank == 0:
            print(json.dumps({"batched": run_batched(args, sg, torch)}), flush=True)
        return
    ctx = sg.spai_ctx_create(stream.cuda_stream, 0)
    fp64_tflops = max(sg.spai_measure_fp64_rate(ctx) for _ in range(3))
    fp32_tflops = max(sg.spai_measure_fp32_rate(ctx) for _ in range(3))

    sweep = Sweep(sg, torch, ctx, w, workers=args.workers)
    sweep.profile(1)  # the warm-up also fills the profiler's pools of CUDA events
    for _ in range(args.warmup):
        sweep.step()
    sweep.solves, sweep.iters = 0, []

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    sweep.profile(1)  # clears the warm-up's totals
    l0 = sg.spai_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        sweep.step()
    for wk in sweep.workers:  # the workers' streams end before e1
        ev = torch.cuda.Event()
        ev.record(wk.stream)
        stream.wait_event(ev)
    e1.record(stream)
    barrier()
    launches = sg.spai_launch_count() - l0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    prof_all = sweep.profile_entries()
    sweep.profile(0)
    prof = [f for f in prof_all if not f["name"].startswith("idle:")]
    idle = sorted(((f["name"][5:], f["ms"]) for f in prof_all if f["name"].startswith("idle:")),
                  key=lambda x: -x[1])
    solves = sweep.solves
    iters = list(sweep.iters)
    t_local = ms / 1e3
    t_max, total_solves = aggregate_replicas(dist, torch, "cuda", t_local, solves)
    value = total_solves / t_max

    def timed_sweep(fp32_roofs=False, **kw):
        """The sweep of the headline with other factor / solve precisions: warm-up, then the
        same number of timed steps (device events, max over ranks).  fp32_roofs: the FP32
        kernel families of the timed steps (the column problems of FP32 builds, the FP32
        operator products) against the FP32 ALU roof."""
        sw = Sweep(sg, torch, ctx, w, workers=args.workers, **kw)
        if fp32_roofs:
            sw.profile(1)  # the warm-up fills the profiler's pools of CUDA events
        for _ in range(max(1, args.warmup)):
            sw.step()
        sw.solves, sw.iters, sw.cycles = 0, [], []
        if fp32_roofs:
            sw.profile(1)  # clears the warm-up's totals
        barrier()
        m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        m0.record(stream)
        for _ in range(args.steps):
            sw.step()
        for wk in sw.workers:
            ev = torch.cuda.Event()
            ev.record(wk.stream)
            stream.wait_event(ev)
        m1.record(stream)
        barrier()
        mt = m0.elapsed_time(m1) / 1e3
        if dist is not None:
            t = torch.tensor([mt], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            mt = t.item()
        out = {"value": sw.solves * world / mt, "unit": UNIT, "ms_per_step": 1e3 * mt / args.steps,
               "gmres_iterations": {"mean": float(np.mean(sw.iters)), "min": int(min(sw.iters)),
                                    "max": int(max(sw.iters))},
               "cycles": {"mean": float(np.mean(sw.cycles)), "max": int(max(sw.cycles))}}
        if fp32_roofs:
            fams = [f for f in sw.profile_entries() if not f["name"].startswith("idle:")]
            sw.profile(0)
            tot = sum(f["ms"] for f in fams) or 1.0
            roofs = {}
            for f in fams:
                if f["name"] in ("spai_columns", "spmm32_A", "spmm32_P") and f["ms"] > 0:
                    r = roofline_entry(f, n=w.n, s=int(w.B.shape[1]), fp32_probe=fp32_tflops, unit="fp32")
                    roofs[f["name"]] = {"launches": f["launches"], "ms": round(f["ms"], 3),
                                        "share": round(f["ms"] / tot, 4), "bound": r["bound"],
                                        "achieved": round(r["achieved"], 3), "unit": r["unit"],
                                        "frac": round(r["frac"], 4), "alu_frac": round(r["alu_frac"], 4)}
            out["kernels_fp32"] = roofs
        sw.close()
        return out

    # the sweep in mixed precision (north star (1)): SPAI build / update in FP32 with FP32
    # factors, the operator A P applied in FP32 inside each restart cycle, FP64 basis,
    # Gram-Schmidt, projected least squares and true residual, FP64 refinement across cycles
    mixed = None
    fp32_factors = None
    if not args.no_mixed:
        mixed = timed_sweep(fp32_roofs=True, prec=sg.PREC_FP32 | sg.LS_NORMAL, solve_precision=sg.SOLVE_MIXED)
        mixed.update({"dtype": "f32 SPAI factors (column problems by their normal equations) and f32 operator "
                               "products, f64 basis/Gram-Schmidt/least squares/true residual (iterative refinement)",
                      "vs_plain_fp64": None})
        fp32_factors = timed_sweep(prec=sg.PREC_FP32)
        fp32_factors["note"] = ("FP32 SPAI factors applied with FP64 products and sums, FP64 solve: the "
                                "factor precision alone")

    # the same FP64 sweep with each solve started from the worker's previous solution of
    # the same shift (every system has the same B; neighbouring p have close solutions):
    # same true-residual tolerance, fewer iterations
    # block GCRO (the paper's solver) with each worker's recycled space along its parameters
    gcro = None
    if not args.no_mixed:
        gcro = timed_sweep(gcro_kmax=args.gcro_kmax)
        gcro["note"] = (f"FP64 as the headline; block GCRO, each worker carrying a recycled space of "
                        f"{args.gcro_kmax} columns per shift (its latest solutions of the shift), cleared every step")
        gcro_mixed = timed_sweep(gcro_kmax=args.gcro_kmax, prec=sg.PREC_FP32 | sg.LS_NORMAL,
                                 solve_precision=sg.SOLVE_MIXED)
        gcro["mixed_precision"] = {k: gcro_mixed[k] for k in ("value", "ms_per_step", "gmres_iterations", "cycles")}
    warm = None
    if not args.no_mixed:
        warm = timed_sweep(warm=True)
        warm["note"] = ("FP64 as the headline; each solve's initial guess is the same worker's previous "
                        "solution of the same shift (the workers take every 4th parameter), not zero")

    # the dominant kernels once more with one solve at a time (no other stream sharing the
    # GPU): their own speed, beside the timed region's contended launch durations
    iso_prof = None
    if rank == 0 and args.workers > 1:
        s1 = Sweep(sg, torch, ctx, w, workers=1)
        s1.step()
        s1.profile(1)
        s1.step()
        iso_prof = [f for f in s1.profile_entries() if not f["name"].startswith("idle:")]
        s1.profile(0)
        s1.close()

    # end-to-end through the C ABI with pinned host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        hs = Sweep(sg, torch, ctx, w, host_inputs=True, workers=args.workers)
        hs.step()  # warm-up
        hs.solves = 0
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            hs.step()
        barrier()
        dt = time.perf_counter() - t0
        if dist is not None:
            t = torch.tensor([dt], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = t.item()
        e2e = {"value": total_solves / dt, "unit": UNIT, "h2d_bytes_per_step": hs.h2d_bytes(),
               "d2h_bytes_per_step": hs.d2h_bytes()}
        hs.close()

    # block GMRES with 8 RHS against 8 single-RHS solves (the paper's block vs non-block)
    bvs = None
    order = None
    if rank == 0 and world == 1 and not args.no_mixed:
        bvs = run_block_vs_single(sg, torch, ctx, w)
        order = run_update_order(sg, torch, ctx, w)
    adaptive = None
    if rank == 0 and world == 1 and not args.no_adaptive:
        adaptive = run_adaptive(sg, torch, ctx, w)
    # many small systems: batched build and lockstep solves
    batched = None
    if rank == 0 and world == 1 and not args.no_batched:
        batched = run_batched(args, sg, torch)
    # the headline's sweep through the server at saturation, beside the plain FP64 sweep
    served_cap = None
    if rank == 0 and world == 1 and not args.no_served_sweep:
        served_cap = run_served_sweep(args, sg, torch, w, min(args.steps, 5))
        served_cap["vs_plain_fp64"] = served_cap["value"] / value
    if mixed is not None:
        mixed["vs_plain_fp64"] = mixed["value"] / value
    # served (continuous admission, update routing, FP32 factors) vs FIFO plain FP64
    serving = None
    if rank == 0 and world == 1 and not args.no_serve:
        serving = run_serving(args, sg, torch)
    large = None
    if rank == 0 and world == 1 and not args.no_large:
        large = run_large(args, sg, torch)

    if rank == 0:
        total_ms = sum(f["ms"] for f in prof) or 1.0
        dom = max(prof, key=lambda f: f["ms"])
        roofline = roofline_entry(dom, n=w.n, s=int(w.B.shape[1]), fp64_probe=fp64_tflops)
        if args.workers > 1:
            roofline["note"] = (f"launch durations of the timed region, where {args.workers} solves share the "
                                f"GPU at a time; roofline_isolated times the same family alone")
        roofline_iso = None
        if iso_prof:
            same = [f for f in iso_prof if f["name"] == dom["name"]]
            if same:
                roofline_iso = roofline_entry(same[0], n=w.n, s=int(w.B.shape[1]), fp64_probe=fp64_tflops)
                roofline_iso["note"] = ("same kernel family, one extra step with a single worker after the "
                                        "timed region (no concurrent stream)")
        kernels = {}
        for f in sorted(prof, key=lambda f: -f["ms"]):
            r = roofline_entry(f, n=w.n, s=int(w.B.shape[1]))
            kernels[f["name"]] = {
                "launches": f["launches"], "ms": round(f["ms"], 3), "share": round(f["ms"] / total_ms, 4),
                "tflops": round(f["flops"] / (f["ms"] * 1e-3) / 1e12, 4) if f["ms"] else 0,
                "gbs": round(f["bytes"] / (f["ms"] * 1e-3) / 1e9, 1) if f["ms"] else 0,
                "bound": r["bound"], "frac": None if r["frac"] is None else round(r["frac"], 4)}
        # order: the contract's keys, then the detail, then (at the end of the line, where a
        # truncated log still shows them) the comparisons the workload is about
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {**workload_config(w, nnz_expected),
                                            "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                                            "workers": args.workers},
            "gpu_launches": int(launches), "clocks": clk, "fp64_tflops_measured": fp64_tflops,
            "fp32_tflops_measured": fp32_tflops,
            "gmres_iterations": {"mean": float(np.mean(iters)), "min": int(min(iters)),
                                 "max": int(max(iters))},
            "kernels": kernels,
            # a worker stream's time with none of its kernels running (mean over the workers),
            # by the kernel family that followed
            "idle_ms": {"total": round(sum(v for _, v in idle), 3),
                        **{k: round(v, 3) for k, v in idle[:8]}},
            "large": large, "batched": batched, "adaptive": adaptive, "update_order": order,
            "block_vs_single_rhs": bvs, "warm_start": warm, "gcro": gcro, "fp32_factors": fp32_factors,
            "serving": serving,
            "cpu_baseline": cpu, "e2e": e2e, "roofline": roofline, "roofline_isolated": roofline_iso,
            "mixed_precision": mixed, "served_capacity": served_cap,
        }
        print(json.dumps(line), flush=True)
    sweep.close()
    sg.spai_ctx_destroy(ctx)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
