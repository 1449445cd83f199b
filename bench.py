"""Benchmark of the MiniFE CG hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step is one pass of the whole path on one synthetic problem: mesh
generation -> CSR assembly with Dirichlet rows -> conversion to the solver
format (paper Sec. 3.1 converts at CG start) -> fused CG to ||r||/||b|| <= 1e-10.
The workload is the paper's problem at Nx = Ny = Nz = 256 (257^3 = 16,974,593
rows, 454,756,609 stored entries), FP64.

Reported (one JSON line on rank 0):
  value        CG time to relative residual 1e-10 (s), mean over the K timed
               steps, max over ranks (CUDA events on the solver's stream)
  ms_per_step  the whole step (mesh + assembly + conversion + CG)
  e2e          the same solve through the Python API with host buffers: the
               boundary data copied in from pinned memory and the solution
               copied out, every step, wall time per step
  roofline     the fused CG kernel against the FP64 pipe and HBM (per-launch
               algorithmic bytes and FLOPs / its CUDA-event time)
  spmv         stand-alone SpMV GB/s of each storage format (the paper's
               CRS vs BCRS comparison) against the measured HBM peak
  mixed        the mixed-precision form on the same system (FP32 values,
               FP32 CG with FP64 reliable updates): time to 1e-10 and its
               speedup over the FP64 solve, with the solutions' difference
  mixed_n400   the N = 400 configuration: FP64 CG vs the mixed solver with FP32
               and with BF16 values, times, steps, true residuals and errors
  single_reduction  the Chronopoulos-Gear CG (one grid reduction per step) on
               the same system, and both CG forms on the N = 30 mesh
  matrix_free  the same system and CG with the operator applied from the
               brick element's Kronecker structure (no stored matrix): time to
               1e-10, steps, difference from the assembled solution, and the
               stand-alone operator pass against the FP64 pipe
  cpu_baseline the CPU oracle, single core, on a bounded sample of the same
               workload (a few CG iterations of the N = 256 system), scaled
               to the solve's iteration count
  cpu_parallel the paper's CG (CRS and variable-length BCRS) with OpenMP on
               all host cores, on the same system, sampled and scaled alike
With --gpus N > 1 (torchrun) every rank solves its own copy (replicas,
weak scaling); the path needs no collective on one mesh per GPU.
``--impl reference`` times the CPU oracle (the only reference that exists
for this paper) on the same workload and metric.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CG time-to-rel-residual 1e-10 (s)"
TOL = 1e-10
MAXIT = 5000
# CG steps to 1e-10 for the N=256 problem from x0 = 0, as counted by the
# fused CG on the GPU (the oracle's count agrees within one step wherever
# both run to the end); the reference arm scales its per-step time by it.
ITERS_TO_TOL = {256: 508}
FP64_PEAK_TFLOPS = 1.25   # nominal dense FP64 of a GB300 (2 FMA/clk/SM x 152 SMs x ~2.06 GHz)
# DRAM bytes (read + write) per row of k_cg<bcrs3,f64>: per CG step and for the
# initial residual plus the last x update, from two ncu captures at N=180 where, as at N=256, the CG
# vectors exceed L2 (profiles/k_cg_n180_ncu_traffic.md).  Valid for the kernel
# as captured; set to None when k_cg changes until it is captured again.
K_CG_BCRS3_TRAFFIC_PER_ROW = {"step": 324.4, "init": 262.7}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples (every 200 ms) of the GPU's SM clock and throttle reasons."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                smax.append(float(p[1]))
                power.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def gpu_selector(torch, dev_index: int) -> str:
    try:
        u = str(torch.cuda.get_device_properties(dev_index).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v for v in vis.split(",") if v.strip()]
        return ids[dev_index] if dev_index < len(ids) else str(dev_index)


# ------------------------------------------------------------------ byte / flop models

def cg_iteration_model(fmt: str, m: int, n_slices: int, n_stored: int, nnz: int):
    """Algorithmic bytes and FP64 FMAs of one CG step of the fused kernel.

    Matrix: every stored index and value once (BCRS3: 4 B index + 3 x 8 B
    values per slot, slice pointers; CSR: 12 B per entry + row pointer).
    Vectors (8 B each per row): w = A p reads p once and writes w (16 B);
    r -= a w reads r, w and writes r (24 B); x += a p, p = r + b p read x, p,
    r and write x, p (40 B): 80 B per row.
    FMAs: one per stored value (padding included) + 5 per row (p.w, x, r,
    r.r, p)."""
    if fmt == "bcrs3":
        mat = 28 * n_stored + 8 * (n_slices + 1)
        fma = 3 * n_stored
    elif fmt == "sell":
        mat = 12 * n_stored + 8 * (n_slices + 1)
        fma = n_stored
    else:
        mat = 12 * nnz + 4 * (m + 1)
        fma = nnz
    return mat + 80 * m, fma + 5 * m, mat


def mixed_bytes_model(m: int, n_slices: int, n_stored: int, value: str, inner_steps: int,
                      refinements: int):
    """Algorithmic bytes of a reliable-update mixed solve on BCRS3 matrices.
    Inner FP32 step: the low-precision matrix once (4 B index + 12 B FP32 or
    6 B BF16 values per slot, slice pointers) and 44 B of FP32 vectors
    per row (w = A p: p, w; xs += a p, r -= a w: xs, r, p, w read, xs, r
    written; p = r + b p: p, r read, p written).  Refinement step: the FP64
    matrix once (28 B per slot) and 44 B per row (x += xs: x, xs read, x, xs
    written; r = b - A x: x, b read, r written).  Plus the initial FP64
    residual."""
    vb = 6 if value == "bf16" else 12
    lo = n_stored * (4 + vb) + 8 * (n_slices + 1) + 44 * m
    hi = 28 * n_stored + 8 * (n_slices + 1) + 44 * m
    return inner_steps * lo + (refinements + 1) * hi


def spmv_bytes(fmt: str, m: int, n_slices: int, n_stored: int, nnz: int, vec_bytes: int = 8):
    if fmt == "vbcrs":      # values, jas and offsets per segment, the segment row pointer
        return 8 * nnz + 4 * n_stored + 4 * (n_stored + 1) + 4 * (m + 1) + 2 * vec_bytes * m
    if fmt == "bcrs3":
        return 28 * n_stored + 8 * (n_slices + 1) + 2 * vec_bytes * m
    if fmt == "sell":
        return 12 * n_stored + 8 * (n_slices + 1) + 2 * vec_bytes * m
    return 12 * nnz + 4 * (m + 1) + 2 * vec_bytes * m


# ------------------------------------------------------------------ CPU oracle sample

def oracle_setup_seconds(sysm, repeats: int = 3) -> float:
    """Median time of an oracle CG call that takes no step (allocation, first
    touch of its vectors, ||b||, r = b - A x0 and r.r): the part of every call
    that does not scale with the step count."""
    import oracle
    ts = []
    for _ in range(repeats):
        t = time.perf_counter()
        oracle.cg(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"], tol=0.0, maxit=0)
        ts.append(time.perf_counter() - t)
    return statistics.median(ts)


def cpu_oracle_sample(n: int, iters_sample: int, iters_to_tol: int):
    """Oracle (single core) on the N-mesh: build the system (untimed setup),
    time a call that takes no step and one that takes `iters_sample` steps;
    the full solve is modelled as setup + iters_to_tol x per-step cost, the
    same model the reference arm uses.  Returns the baseline entry and the
    oracle's system (reused by the multi-core leg)."""
    import oracle
    t0 = time.perf_counter()
    sysm = oracle.build_system(n, n, n)
    build = time.perf_counter() - t0
    setup = oracle_setup_seconds(sysm)
    t1 = time.perf_counter()
    oracle.cg(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"], tol=0.0, maxit=iters_sample)
    dt = time.perf_counter() - t1
    per_it = (dt - setup) / iters_sample
    return {"value": setup + per_it * iters_to_tol, "unit": "s", "cores": 1, "kind": "oracle",
            "s_per_iteration": round(per_it, 5), "setup_s": round(setup, 4),
            "sample": (f"oracle (plain C, 1 thread) on the N={n} system: one call of "
                       f"{iters_sample} CG iterations ({dt:.1f} s) less the call setup "
                       f"({setup:.2f} s: vectors, r = b - A x0) gives {per_it:.4f} s/iteration; "
                       f"value = setup + {iters_to_tol} iterations; its "
                       f"mesh+pattern+assembly took {build:.1f} s (untimed)")}, sysm


def cpu_oracle_full_solve(n: int, repeats: int = 3):
    """The oracle's whole solve (CG from x0 = 0 to 1e-10) on the N-mesh, timed
    in full: median of `repeats` runs."""
    import oracle
    sysm = oracle.build_system(n, n, n)
    ts, its = [], None
    for _ in range(repeats):
        t = time.perf_counter()
        _, its, rel, st = oracle.cg(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"],
                                    tol=TOL, maxit=MAXIT)
        ts.append(time.perf_counter() - t)
    return {"value": round(statistics.median(ts), 5), "unit": "s", "cores": 1, "kind": "oracle",
            "iterations": its, "status": st, "runs_s": [round(t, 5) for t in ts],
            "sample": f"oracle CG on the N={n} mesh from x0=0 to 1e-10, timed in full, "
                      f"median of {repeats} runs"}


def cpu_parallel_sample(sysm, n: int, iters_sample: int, iters_to_tol: int):
    """The paper's CG on all host cores (OpenMP, CRS and the paper's
    variable-length BCRS) on the oracle's system: `iters_sample` CG steps
    timed inside the C code, scaled to the iteration count to 1e-10."""
    import oracle
    out = {"unit": "s", "kind": "openmp", "cores_online": os.cpu_count()}
    t0 = time.perf_counter()
    ptr, jas, off = oracle.csr_to_bcrs(sysm["row_ptr"], sysm["cols"])
    conv = time.perf_counter() - t0
    for fmt, args in (("csr", (sysm["row_ptr"], sysm["cols"], sysm["vals"])),
                      ("bcrs", (ptr, jas, sysm["vals"]))):
        kw = {"offsets": off} if fmt == "bcrs" else {}
        _, it, _, st, sec, thr = oracle.omp_cg(fmt, sysm["b"], *args, tol=0.0, maxit=iters_sample, **kw)
        per_it = sec / max(it, 1)
        out[fmt] = {"value": round(per_it * iters_to_tol, 4), "s_per_iteration": round(per_it, 5),
                    "threads": thr}
        out["cores"] = thr
    out["sample"] = (f"OpenMP CG (gcc -O3 -fopenmp, {out['cores']} threads) on the oracle's N={n} "
                     f"system, {iters_sample} steps per storage form timed and scaled to "
                     f"{iters_to_tol} steps; BCRS index build {conv:.1f} s (untimed)")
    return out


# ------------------------------------------------------------------ reference arm

def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    import oracle
    n = args.n
    iters_to_tol = ITERS_TO_TOL.get(n, int(round(2.08 * n)))
    if args.ref_iters is None:   # at least 40 timed iterations, as the cpu_baseline leg's sample
        args.ref_iters = max(2, -(-40 // max(1, args.steps)))
    t0 = time.perf_counter()
    sysm = oracle.build_system(n, n, n)
    setup = time.perf_counter() - t0
    setup_s = oracle_setup_seconds(sysm)
    per_step, per_it_steps = [], []
    for i in range(args.warmup + args.steps):
        t1 = time.perf_counter()
        oracle.cg(sysm["row_ptr"], sysm["cols"], sysm["vals"], sysm["b"], tol=0.0,
                  maxit=args.ref_iters)
        dt = time.perf_counter() - t1
        if i >= args.warmup:
            per_step.append(dt)
            per_it_steps.append((dt - setup_s) / args.ref_iters)
    per_it = statistics.mean(per_it_steps)
    value = setup_s + per_it * iters_to_tol
    spread = (max(per_it_steps) - min(per_it_steps)) / per_it
    sample = (f"each step: one oracle call of {args.ref_iters} CG iterations on the N={n} system "
              f"less the call setup ({setup_s:.2f} s, measured before the steps): "
              f"{per_it:.4f} s/iteration over {args.steps * args.ref_iters} timed iterations "
              f"(spread over steps {100 * spread:.1f} %), 1 thread; value = setup + "
              f"{iters_to_tol} iterations, the model the bench's cpu_baseline uses; oracle "
              f"mesh+pattern+assembly {setup:.1f} s (untimed)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(per_step) * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args),
            "cpu_baseline": {"value": value, "unit": "s", "cores": 1, "kind": "oracle",
                             "s_per_iteration": round(per_it, 5),
                             "per_step_spread": round(spread, 4), "sample": sample},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def max_over_ranks(values, device):
    """Element-wise maximum of `values` over the ranks of the default process
    group (the slowest replica sets every time in the line)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def config_dict(args):
    n = args.n
    m = (n + 1) ** 3
    nnz = (3 * n + 1) ** 3
    return {"workload": (f"MiniFE heat conduction, unit cube, N={n} ({n + 1}^3 = {m:,} rows, "
                         f"{nnz:,} stored entries), FP64, {args.format.upper()} solver format, "
                         f"unpreconditioned CG from x0=0 to ||r||/||b|| <= 1e-10"),
            "nx": n, "ny": n, "nz": n, "format": args.format, "tol": TOL,
            "l2": "inputs larger than L2 (the matrix alone is >4 GB)"}


# ------------------------------------------------------------------ our arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", "--elements", dest="n", type=int, default=256,
                    help="elements per axis (--elements: the same, a name torchrun does not take for its own)")
    ap.add_argument("--format", choices=["csr", "sell", "bcrs3"], default="bcrs3")
    ap.add_argument("--cpu-iters", type=int, default=40, help="oracle CG iterations in the CPU sample")
    ap.add_argument("--cpu-parallel-iters", type=int, default=40,
                    help="OpenMP CG iterations per storage form in the multi-core CPU sample (0: skip)")
    ap.add_argument("--ref-iters", type=int, default=None,
                    help="oracle CG iterations per reference step (default: enough for 40 timed "
                         "iterations over the timed steps, the cpu_baseline leg's sample)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-spmv", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-warm-start", action="store_true", help="skip the learned warm-start leg")
    ap.add_argument("--no-sr", action="store_true", help="skip the single-reduction CG legs")
    ap.add_argument("--no-n400", action="store_true", help="skip the N=400 mixed-precision leg")
    ap.add_argument("--no-matrix-free", action="store_true", help="skip the matrix-free leg")
    ap.add_argument("--batch-size", type=int, default=64)
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    import paper_1505_08023_gb300.fe as fe

    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    hbm_peak, peak_kind = load_peaks()

    n = args.n
    s = fe.System(n, device=dev)
    m = s.m
    x = torch.zeros(m, dtype=torch.float64, device=dev)
    EV = lambda: torch.cuda.Event(enable_timing=True)
    state = {}

    def step():
        e = [EV() for _ in range(5)]
        e[0].record()
        s.generate_mesh()
        e[1].record()
        s.assemble(keep_workspace=True)
        e[2].record()
        A = s.convert(args.format, "f64")
        e[3].record()
        if "work" not in state:
            state["work"] = fe.cg_workspace(A, dev)
        x.zero_()
        res = fe.fe_cg_solve(A.desc, s.b, x, TOL, MAXIT, state["work"], check=False)
        e[4].record()
        state["A"] = A
        return e, res

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(gpu_selector(torch, local))
    sampler.start()
    time.sleep(0.3)
    t_wall = time.perf_counter()
    records = []
    for _ in range(args.steps):
        records.append(step())
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - t_wall
    clocks = sampler.stop()

    phases = {"mesh": [], "assembly": [], "convert": [], "cg": [], "step": []}
    iters, statuses = [], set()
    for e, res in records:
        phases["mesh"].append(e[0].elapsed_time(e[1]))
        phases["assembly"].append(e[1].elapsed_time(e[2]))
        phases["convert"].append(e[2].elapsed_time(e[3]))
        phases["cg"].append(e[3].elapsed_time(e[4]))
        phases["step"].append(e[0].elapsed_time(e[4]))
        iters.append(res.iterations)
        statuses.add(res.status)
    cg_ms = statistics.mean(phases["cg"])
    step_ms = statistics.mean(phases["step"])
    if world > 1:
        cg_ms, step_ms = max_over_ranks([cg_ms, step_ms], dev)

    A = state["A"]
    it = statistics.mean(iters)
    tr = fe.fe_true_relres(A.desc, s.b, x, fe.resid_workspace(dev))
    byte_it, fma_it, mat_bytes = cg_iteration_model(args.format, m, s.sizes.n_slices,
                                                     A.desc.n_stored, s.sizes.nnz)
    # one launch: the initial residual (one matrix pass + b, x, r, p) plus `it` steps
    launch_bytes = it * byte_it + mat_bytes + 40 * m + 24 * m   # + the last x update (x, p in, x out)
    launch_fma = it * fma_it + fma_it - 5 * m + 2 * m
    t_launch = cg_ms * 1e-3
    hbm_ach = launch_bytes / t_launch / 1e9
    fp64_ach = 2 * launch_fma / t_launch / 1e12
    hbm_floor = launch_bytes / (hbm_peak * 1e9)
    alu_floor = 2 * launch_fma / (FP64_PEAK_TFLOPS * 1e12)
    bound = "alu" if alu_floor > hbm_floor else "hbm"
    traffic = None
    if args.format == "bcrs3" and K_CG_BCRS3_TRAFFIC_PER_ROW:
        t = K_CG_BCRS3_TRAFFIC_PER_ROW
        traffic = int((it * t["step"] + t["init"]) * m)
    roof_hbm = {"bound": "hbm", "achieved": round(hbm_ach, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(hbm_ach / hbm_peak, 4), "traffic": traffic,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"}
    roof_alu = {"bound": "alu", "achieved": round(fp64_ach, 4), "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": round(fp64_ach / FP64_PEAK_TFLOPS, 4), "traffic": traffic,
                "peak_source": "nominal FP64 (2 DFMA/clk/SM x 152 SMs); probe measured 1.26"}
    roofline = dict(roof_alu if bound == "alu" else roof_hbm)
    roofline.update({"kernel": f"k_cg<{args.format},f64>",
                     "algorithmic_bytes_per_launch": int(launch_bytes),
                     "fp64_flops_per_launch": int(2 * launch_fma),
                     "other": roof_hbm if bound == "alu" else roof_alu})

    # ---- mixed-precision form on the same system (FP32 and BF16 values, reliable updates)
    mixed = None
    if not args.no_mixed:
        x64_ref = x.clone()                        # the FP64 solve's solution
        A64 = state["A"]
        acc = MixedAccuracy(fe, torch, A64, s.b, x64_ref, n, dev)
        mixed = {}
        for v in ("f32", "bf16"):
            Alo = s.convert(args.format, v)
            mwork = fe.mixed_workspace(Alo, dev)
            xm = torch.zeros(m, dtype=torch.float64, device=dev)

            def mixed_solve():
                xm.zero_()
                a, b = EV(), EV()
                a.record()
                r = fe.fe_cg_solve_mixed(A64.desc, Alo.desc, s.b, xm, TOL, fe.FE_MIXED_RELIABLE, 200,
                                         0.1, MAXIT, mwork, check=False)
                b.record()
                return a, b, r

            for _ in range(args.warmup):
                mixed_solve()
            torch.cuda.synchronize()
            recs = [mixed_solve() for _ in range(args.steps)]
            torch.cuda.synchronize()
            mt = statistics.mean(a.elapsed_time(b) for a, b, _ in recs)
            r = recs[-1][2]
            err = float(torch.linalg.norm(xm - x64_ref) / torch.linalg.norm(x64_ref))
            entry = {"value": round(mt * 1e-3, 6), "unit": "s", "values": v,
                     "mode": "reliable updates (FP32 CG, FP64 residual/update/dots), delta 0.1",
                     "speedup_vs_fp64": round(cg_ms / mt, 3), "fp32_iterations": r.inner_iterations,
                     "refinement_steps": r.outer_iterations, "relres_true": r.relres,
                     "status": r.status, "rel_diff_vs_fp64_solution": err,
                     "ms_per_fp32_iteration": round(mt / max(r.inner_iterations, 1), 4),
                     "accuracy": acc.entry(xm)}
            if args.format == "bcrs3":
                byts = mixed_bytes_model(m, s.sizes.n_slices, Alo.desc.n_stored, v,
                                         r.inner_iterations, r.outer_iterations)
                ach = byts / (mt * 1e-3) / 1e9
                entry["roofline"] = {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm_peak,
                                     "unit": "GB/s", "frac": round(ach / hbm_peak, 4),
                                     "algorithmic_bytes": int(byts),
                                     "model": "inner FP32 steps + FP64 refinement passes"}
            if v == "f32":
                mixed.update(entry)       # the FP32-value form is the leg's headline
            else:
                mixed["bf16"] = entry
            s._formats.pop((args.format, v), None)
            del Alo, mwork, xm
            torch.cuda.empty_cache()
        mixed["fp64_accuracy"] = acc.entry(x64_ref)
        del acc
        torch.cuda.empty_cache()

    # ---- single-reduction CG (Chronopoulos-Gear): the same system, and the N=30 mesh
    single_red = None
    if not args.no_sr:
        A64 = state["A"]
        srwork = fe.sr_workspace(A64, dev)
        xs = torch.zeros(m, dtype=torch.float64, device=dev)

        def sr_solve(Am, bm, xm, wk):
            xm.zero_()
            a, b = EV(), EV()
            a.record()
            r = fe.fe_cg_solve_sr(Am.desc, bm, xm, TOL, MAXIT, wk, check=False)
            b.record()
            return a, b, r

        for _ in range(args.warmup):
            sr_solve(A64, s.b, xs, srwork)
        torch.cuda.synchronize()
        recs = [sr_solve(A64, s.b, xs, srwork) for _ in range(args.steps)]
        torch.cuda.synchronize()
        st_ms = statistics.mean(a.elapsed_time(b) for a, b, _ in recs)
        r = recs[-1][2]
        single_red = {"value": round(st_ms * 1e-3, 6), "unit": "s", "iterations": r.iterations,
                      "status": r.status, "speedup_vs_textbook": round(cg_ms / st_ms, 3),
                      "rel_diff_vs_textbook_solution":
                          float(torch.linalg.norm(xs - x) / torch.linalg.norm(x))}
        del srwork, xs
        # the small mesh (N = 30, 29,791 rows): L2-resident, barrier-bound
        small = fe.System(30, device=dev).build()
        As = small.matrix(args.format, "f64")
        xsm = torch.zeros(small.m, dtype=torch.float64, device=dev)
        out = {}
        def form(f):
            return lambda A_, b_, x_, t_, k_, w_, check=False: fe.fe_cg_solve_form(
                A_, b_, x_, t_, k_, f, w_, check=check)
        # fe_cg_solve picks the matrix-resident form on this mesh (one slice per
        # warp, FP64 BCRS3); the other textbook forms for comparison
        cw = fe.cg_workspace(As, dev)
        for name, fn, wk in (("textbook", fe.fe_cg_solve, cw),
                             ("textbook_two_phase", form(fe.FE_CG_TWO_PHASE), cw),
                             ("textbook_three_phase", form(fe.FE_CG_THREE_PHASE), cw),
                             ("single_reduction", fe.fe_cg_solve_sr, fe.sr_workspace(As, dev))):
            ts = []
            for _ in range(args.warmup + args.steps):
                xsm.zero_()
                a, b = EV(), EV()
                a.record()
                r = fn(As.desc, small.b, xsm, TOL, MAXIT, wk, check=False)
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            t_ms = statistics.mean(ts[args.warmup:])
            out[name] = {"ms": round(t_ms, 4), "iterations": r.iterations, "status": r.status,
                         "us_per_iteration": round(1e3 * t_ms / max(r.iterations, 1), 2)}
        single_red["n30"] = out
        del small, As, xsm
        torch.cuda.empty_cache()

    # ---- matrix-free operator: the same system and CG without a stored matrix
    matrix_free = None
    if not args.no_matrix_free:
        matrix_free = run_matrix_free(args, fe, torch, dev, EV, n, s, x, cg_ms)

    # ---- batched form: 64 cubic meshes N ~ U{32..128}, random face data
    batched = None
    if not args.no_batched and world == 1:
        batched = run_batched(args, fe, torch, dev, EV)
    warm = None
    if not args.no_warm_start and world == 1:
        warm = run_warm_start(args, fe, torch, dev, EV)
        torch.cuda.empty_cache()

    # ---- the N = 400 mixed-precision configuration (FP32 and BF16 values)
    n400 = None
    if not args.no_n400 and world == 1:
        n400 = run_n400(args, fe, torch, dev, EV)

    # ---- e2e: host boundary data in, host solution out, through the Python API
    e2e = None
    if True:
        import fe_inputs
        fv_host = torch.from_numpy(exact_minife_faces(n)).pin_memory()
        x_host = torch.empty(m, dtype=torch.float64).pin_memory()
        fv_dev = torch.empty(fv_host.numel(), dtype=torch.float64, device=dev)
        s.face_vals = fv_dev

        def e2e_step():
            fv_dev.copy_(fv_host, non_blocking=True)
            s.generate_mesh()
            s.assemble(keep_workspace=True)
            A2 = s.convert(args.format, "f64")
            x.zero_()
            r = fe.fe_cg_solve(A2.desc, s.b, x, TOL, MAXIT, state["work"], check=False)
            x_host.copy_(x, non_blocking=True)
            torch.cuda.current_stream().synchronize()
            return r

        for _ in range(max(1, args.warmup)):
            e2e_step()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            r2 = e2e_step()
        e2e_s = (time.perf_counter() - t0) / args.steps
        # same problem as the device-resident run: identical solution bits
        same = bool(torch.equal(x_host, x.cpu()))
        e2e = {"value": round(e2e_s, 5), "unit": "s",
               "h2d_bytes_per_step": fv_host.numel() * 8, "d2h_bytes_per_step": m * 8,
               "what": "boundary face data H2D, mesh, assembly, conversion, CG, solution D2H; "
                       "wall time per step", "iterations": r2.iterations,
               "solution_matches_device_run": same}
        s.face_vals = None

    # ---- stand-alone SpMV of each format (paper Fig 3.1 vs Fig 3.2/3.3)
    spmv = None
    if not args.no_spmv:
        spmv = {}
        xv = torch.rand(m, dtype=torch.float64, device=dev)
        yv = torch.empty_like(xv)
        flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
        for fmt in ["csr", "sell", "bcrs3", "vbcrs"]:
            Af = s.matrix(fmt, "f64")
            ts = []
            for r in range(7):
                flush.zero_()
                a, b = EV(), EV()
                a.record()
                fe.fe_spmv(Af.desc, xv, yv)
                b.record()
                torch.cuda.synchronize()
                if r >= 2:
                    ts.append(a.elapsed_time(b))
            t = statistics.median(ts)
            byts = spmv_bytes(fmt, m, s.sizes.n_slices, Af.desc.n_stored, s.sizes.nnz)
            spmv[fmt] = {"ms": round(t, 4), "algorithmic_gb": round(byts / 1e9, 4),
                         "gbs": round(byts / t / 1e6, 1), "frac_hbm": round(byts / t / 1e6 / hbm_peak, 4),
                         "fp64_tflops": round(2 * (3 * Af.desc.n_stored if fmt == "bcrs3" else
                                                   (Af.desc.n_stored if fmt == "sell" else s.sizes.nnz))
                                              / t / 1e9, 4)}
            if fmt == "vbcrs":
                spmv[fmt]["segments"] = int(Af.desc.n_stored)
                spmv[fmt]["what"] = "the paper's BCRS as printed: ptr, jas, offsets over the CRS values"
            if fmt != args.format:
                s._formats.pop((fmt, "f64"), None)
            del Af
        del flush
        torch.cuda.empty_cache()

    launches_per_step = 7   # mesh 1, assembly 2, slice plan 2, fill 1, CG 1 (timed FP64 steps)

    if rank == 0:
        cpu = cpu_par = cpu_n30 = None
        if world == 1 and not args.no_cpu_baseline:
            cpu_n30 = cpu_oracle_full_solve(30)
            cpu, sysm = cpu_oracle_sample(n, args.cpu_iters, int(round(it)))
            if args.cpu_parallel_iters > 0:
                cpu_par = cpu_parallel_sample(sysm, n, args.cpu_parallel_iters, int(round(it)))
            del sysm
        line = {"metric": METRIC, "value": round(cg_ms * 1e-3, 6), "unit": "s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(step_ms, 3), "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": config_dict(args),
                "iterations": it, "relres_true": tr, "status": sorted(statuses),
                "cg_ms_per_iteration": round(cg_ms / max(it, 1), 4),
                "phase_ms": {k: round(statistics.mean(v), 3) for k, v in phases.items()},
                "roofline": roofline, "cpu_baseline_n30": cpu_n30, "mixed": mixed, "mixed_n400": n400, "single_reduction": single_red,
                "matrix_free": matrix_free,
                "batched": batched, "warm_start": warm, "spmv": spmv, "e2e": e2e,
                "cpu_baseline": cpu, "cpu_parallel": cpu_par,
                "clocks": clocks, "gpu_launches": launches_per_step * args.steps,
                "wall_s_timed_region": round(wall, 3)}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def matrix_free_ops(n: int):
    """FP64 pipe operations (add, mul and FMA one each) of the matrix-free
    path on the N^3 cube: the operator takes 9 per interior row (plane sums
    Sx, Sy and D = Sx above + Sx below: 3; P = c3 (Sx + Sy) + c7 D: 3;
    c0 X + c3 D + P(z-1) + P(z+1): 3); a CG step adds the p.w product, the
    x update and the staging of p = r + beta p in phase A (3 per interior
    row; 3 per boundary row in all) and r -= alpha w, r.r in phase B (2 per
    row).  Halo recomputation (Sx of the two halo rows, the 2 extra planes
    per column segment, the 1.33x staged p) is not counted."""
    m = (n + 1) ** 3
    inner = (n - 1) ** 3
    bc = m - inner
    return {"spmv": 9 * inner, "step": 12 * inner + 3 * bc + 2 * m, "init": 10 * inner + 2 * m}


def run_matrix_free(args, fe, torch, dev, EV, n: int, s, x_assembled, cg_ms: float):
    """The N^3 system without a stored matrix: right-hand side from the
    boundary values, CG to 1e-10 (CUDA events around fe_stencil_cg_solve,
    one launch of k_cg_stencil), its difference from the assembled solve, and
    the stand-alone operator pass (L2 flushed between passes)."""
    mf = fe.StencilSystem(n, device=dev).build()
    rhs_diff = float((mf.b - s.b).abs().max())
    xm = torch.zeros(mf.m, dtype=torch.float64, device=dev)
    ts = []
    for i in range(args.warmup + args.steps):
        xm.zero_()
        a, b = EV(), EV()
        a.record()
        r = mf.solve(xm, TOL, MAXIT, check=False)
        b.record()
        torch.cuda.synchronize()
        if i >= args.warmup:
            ts.append(a.elapsed_time(b))
    t_ms = statistics.mean(ts)
    ops = matrix_free_ops(n)
    fp64_ops_peak = FP64_PEAK_TFLOPS * 1e12 / 2       # pipe operations per second
    step_ops = ops["init"] + r.iterations * ops["step"]
    out = {"value": round(t_ms * 1e-3, 6), "unit": "s", "iterations": r.iterations, "status": r.status,
           "ms_per_iteration": round(t_ms / max(r.iterations, 1), 4),
           "speedup_vs_assembled": round(cg_ms / t_ms, 3),
           "rel_diff_vs_assembled_solution": float(torch.linalg.norm(xm - x_assembled) /
                                                   torch.linalg.norm(x_assembled)),
           "max_abs_rhs_diff_vs_assembled": rhs_diff,
           "relres_true": mf.true_relres(xm),
           "roofline": {"bound": "alu", "achieved": round(step_ops / (t_ms * 1e-3) / 1e9, 1),
                        "peak": round(fp64_ops_peak / 1e9, 1), "unit": "GFP64op/s",
                        "frac": round(step_ops / (t_ms * 1e-3) / fp64_ops_peak, 4),
                        "ops_per_interior_row_step": 12, "vector_bytes_per_row_step": 72}}
    yv = torch.empty_like(xm)
    xv = torch.rand(mf.m, dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    sp = []
    for i in range(7):
        flush.zero_()
        a, b = EV(), EV()
        a.record()
        mf.spmv(xv, yv)
        b.record()
        torch.cuda.synchronize()
        if i >= 2:
            sp.append(a.elapsed_time(b))
    t = statistics.median(sp)
    out["spmv"] = {"ms": round(t, 4), "fp64_ops_per_row": 9,
                   "gops": round(ops["spmv"] / t / 1e6, 1),
                   "frac_fp64": round(ops["spmv"] / (t * 1e-3) / fp64_ops_peak, 4),
                   "algorithmic_gb": round(16 * mf.m / 1e9, 4),
                   "gbs": round(16 * mf.m / t / 1e6, 1)}
    del mf, xm, yv, xv, flush
    torch.cuda.empty_cache()
    return out


def lambda_min_cube(n: int) -> float:
    """Smallest eigenvalue of the Dirichlet system of the n^3 box mesh: the
    boundary rows' identity (eigenvalue 1) and the interior block, the Kronecker
    sum of 1D linear-element stiffness and mass, whose smallest eigenvalue is
    3 l(1) m(1)^2 with l(1) = (2/h)(1 - cos pi h), m(1) = (h/3)(2 + cos pi h)."""
    import math
    h = 1.0 / n
    c = math.cos(math.pi * h)
    lam = 3.0 * (2.0 / h) * (1.0 - c) * ((h / 3.0) * (2.0 + c)) ** 2 if n >= 2 else 1.0
    return min(1.0, lam)


class MixedAccuracy:
    """Errors of a solve against x* (the FP64 solve to 1e-13, untimed) and the
    per-form bars: the forward-error bound ||x - x*|| <= (||b - A x|| +
    ||b - A x*||) / lambda_min that every solution meeting the residual test
    obeys, and the regression guard of 20x the FP64 solve's own error."""

    def __init__(self, fe, torch, A64, b, x64, n, dev):
        self.fe, self.torch, self.A64, self.b = fe, torch, A64, b
        self.rwork = fe.resid_workspace(dev)
        self.xs = torch.zeros_like(x64)
        w = fe.cg_workspace(A64, dev)
        fe.fe_cg_solve(A64.desc, b, self.xs, 1e-13, 20000, w, check=False)
        del w
        self.bnorm = float(torch.linalg.norm(b))
        self.xsnorm = float(torch.linalg.norm(self.xs))
        self.rs = fe.fe_true_relres(A64.desc, b, self.xs, self.rwork) * self.bnorm
        self.lam = lambda_min_cube(n)
        self.e64 = float(torch.linalg.norm(x64 - self.xs))

    def entry(self, x):
        e = float(self.torch.linalg.norm(x - self.xs))
        rel_res = self.fe.fe_true_relres(self.A64.desc, self.b, x, self.rwork)
        bound = (rel_res * self.bnorm + self.rs) / self.lam
        return {"rel_error_vs_xstar": e / self.xsnorm,
                "ratio_to_fp64_error": e / self.e64 if self.e64 > 0 else None,
                "forward_error_bound_rel": bound / self.xsnorm,
                "meets_bound": bool(e <= bound), "meets_guard_20x": bool(e <= 20 * self.e64 + 1e-12 * self.xsnorm),
                "relres_true": rel_res,
                "xstar": "FP64 CG to 1e-13 on the same system"}


def run_n400(args, fe, torch, dev, EV, n: int = 400):
    """Mixed precision at N = 400 (401^3 = 64.5M rows, 1.73B stored entries):
    FP64 CG (BCRS3) to 1e-10, then the reliable-update mixed solver with FP32
    and with BF16 values (BCRS3), each to a true relative residual of 1e-10;
    one untimed and one timed solve each (the matrix alone exceeds L2 ~100x).
    Errors are against the FP64 GPU solve (the same solver checked against
    the oracle in the tests); the true residuals come from the FP64 residual
    kernel."""
    hbm_peak, _ = load_peaks()
    s = fe.System(n, device=dev).build()
    A64 = s.matrix("bcrs3", "f64")
    lo = {v: s.matrix("bcrs3", v) for v in ("f32", "bf16")}
    s.cols = s.vals = None           # the CSR copy is no longer needed
    s.coords = None
    torch.cuda.empty_cache()
    m = s.m
    rwork = fe.resid_workspace(dev)
    out = {"workload": f"MiniFE N={n} ({m:,} rows, {s.sizes.nnz:,} stored entries), BCRS3",
           "unit": "s"}
    x64 = torch.zeros(m, dtype=torch.float64, device=dev)
    w64 = fe.cg_workspace(A64, dev)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = EV(), EV()
        a.record()
        r = fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) * 1e-3, r

    def fp64():
        x64.zero_()
        return fe.fe_cg_solve(A64.desc, s.b, x64, TOL, 20000, w64, check=False)

    t, r = timed(fp64)
    acc = MixedAccuracy(fe, torch, A64, s.b, x64, n, dev)
    out["fp64"] = {"value": round(t, 4), "iterations": r.iterations, "status": r.status,
                   "relres_true": fe.fe_true_relres(A64.desc, s.b, x64, rwork),
                   "accuracy": acc.entry(x64)}
    for v, Alo in lo.items():
        xm = torch.zeros(m, dtype=torch.float64, device=dev)
        mw = fe.mixed_workspace(Alo, dev)

        def mixed():
            xm.zero_()
            return fe.fe_cg_solve_mixed(A64.desc, Alo.desc, s.b, xm, TOL, fe.FE_MIXED_RELIABLE, 200,
                                        0.1, 20000, mw, check=False)

        t, r = timed(mixed)
        out[v] = {"value": round(t, 4), "status": r.status, "inner_iterations": r.inner_iterations,
                  "refinement_steps": r.outer_iterations,
                  "relres_true": fe.fe_true_relres(A64.desc, s.b, xm, rwork),
                  "rel_error_vs_fp64": float(torch.linalg.norm(xm - x64) / torch.linalg.norm(x64)),
                  "accuracy": acc.entry(xm),
                  "speedup_vs_fp64": round(out["fp64"]["value"] / t, 3)}
        byts = mixed_bytes_model(m, s.sizes.n_slices, Alo.desc.n_stored, v, r.inner_iterations,
                                 r.outer_iterations)
        out[v]["roofline"] = {"bound": "hbm", "achieved": round(byts / t / 1e9, 1), "peak": hbm_peak,
                              "unit": "GB/s", "frac": round(byts / t / 1e9 / hbm_peak, 4),
                              "algorithmic_bytes": int(byts)}
        del xm, mw
    del s, A64, lo, x64, w64, acc
    torch.cuda.empty_cache()
    return out


def run_warm_start(args, fe, torch, dev, EV, n_eval: int = 50, n_accuracy: int = 2):
    """Learned warm start (N = 128, 129^3 nodes): the committed trained network
    (paper_1505_08023_gb300/weights/warmstart_n128.blob, trained on 2,000 CG
    solutions for face data PCG64(1000, 0..1999)) on held-out face data
    PCG64(2000, 0..n_eval-1).  Per problem: FP64 CG (BCRS3) from x0 = 0, and
    the network's x0 (one fe_warmstart_infer call) checked by its true
    residual (x0 = 0 as the fallback when it is not below 1) then FP64 CG to
    the same tolerance; CUDA events around each, the warm time including
    inference and the check.  On the first n_accuracy problems both solutions
    are compared with x* (the FP64 solve to 1e-13) and their true residuals
    reported."""
    import fe_inputs
    from paper_1505_08023_gb300 import warmstart as ws
    if not os.path.exists(ws.DEFAULT_BLOB):
        return {"unavailable": "no trained network blob"}
    net = ws.TrainedWarmStart(ws.DEFAULT_BLOB, dev)
    N = net.n_nodes - 1
    prob = ws.Problem(N, dev)
    m = prob.sys.m
    rwork = fe.resid_workspace(dev)
    x = torch.zeros(m, dtype=torch.float64, device=dev)
    x0 = torch.empty_like(x)
    lam = lambda_min_cube(N)
    rows, acc = [], []
    for i in range(n_eval):
        prob.set_faces(fe_inputs.face_data(2000, i, N, N, N))
        for _ in range(2 if i == 0 else 1):          # the first problem once untimed
            x.zero_()
            a, b = EV(), EV()
            a.record()
            r0 = fe.fe_cg_solve(prob.A.desc, prob.sys.b, x, TOL, MAXIT, prob.work, check=False)
            b.record()
            a2, b2, c2 = EV(), EV(), EV()
            a2.record()
            net.predict(prob.sys, x0)
            b2.record()
            start_res = fe.fe_true_relres(prob.A.desc, prob.sys.b, x0, rwork)
            fallback = not (start_res < 1.0)
            if fallback:
                x0.zero_()
            r1 = fe.fe_cg_solve(prob.A.desc, prob.sys.b, x0, TOL, MAXIT, prob.work, check=False)
            c2.record()
            torch.cuda.synchronize()
        rows.append((r0.iterations, r1.iterations, a.elapsed_time(b), a2.elapsed_time(c2),
                     a2.elapsed_time(b2), start_res, fallback, r0.status == 0 and r1.status == 0))
        if i < n_accuracy:
            xs = torch.zeros_like(x)
            fe.fe_cg_solve(prob.A.desc, prob.sys.b, xs, 1e-13, MAXIT, prob.work, check=False)
            xsn = float(torch.linalg.norm(xs))
            bn = float(torch.linalg.norm(prob.sys.b))
            rs = fe.fe_true_relres(prob.A.desc, prob.sys.b, xs, rwork) * bn
            entry = {"seed": f"PCG64(2000, {i})"}
            for name, v in (("cold", x), ("warm", x0)):
                tr = fe.fe_true_relres(prob.A.desc, prob.sys.b, v, rwork)
                e = float(torch.linalg.norm(v - xs))
                entry[name] = {"relres_true": tr, "rel_error_vs_xstar": e / xsn,
                               "forward_error_bound_rel": (tr * bn + rs) / lam / xsn}
            acc.append(entry)
    ic = [r[0] for r in rows]
    iw = [r[1] for r in rows]
    tc = [r[2] for r in rows]
    tw = [r[3] for r in rows]
    return {"workload": (f"MiniFE N={N} ({m:,} rows), random face data, {n_eval} held-out problems; "
                         f"FP64 CG (BCRS3) to 1e-10 from x0 = 0 and from the network's x0"),
            "unit": "ms", "samples": n_eval,
            "mean_iterations_cold": statistics.mean(ic), "mean_iterations_warm": statistics.mean(iw),
            "iterations_saved_frac": round(1 - statistics.mean(iw) / statistics.mean(ic), 4),
            "mean_ms_cold": round(statistics.mean(tc), 4),
            "mean_ms_warm_incl_inference": round(statistics.mean(tw), 4),
            "time_saved_frac": round(1 - statistics.mean(tw) / statistics.mean(tc), 4),
            "mean_ms_inference": round(statistics.mean(r[4] for r in rows), 4),
            "mean_start_relres": statistics.mean(r[5] for r in rows),
            "fallbacks": sum(r[6] for r in rows), "all_converged": all(r[7] for r in rows),
            "accuracy": acc,
            "network": {k: net.meta.get(k) for k in ("channels", "n_train", "epochs", "train_seeds")}}


def run_batched(args, fe, torch, dev, EV):
    """64 independent problems (cubic meshes, N ~ U{32..128} from PCG64 seed 0,
    random Dirichlet face data) solved to 1e-10 in one persistent launch, with
    the launch shape chosen by the autotuner and the launch replayed from a
    CUDA graph; against the same systems through fe_cg_solve one by one."""
    import fe_inputs
    from paper_1505_08023_gb300 import autotune
    sizes = [int(n) for n in fe_inputs.batched_sizes(0, args.batch_size)]
    faces = [fe_inputs.face_data(0, i, n, n, n) for i, n in enumerate(sizes)]
    batch = fe.Batch(sizes, faces, "bcrs3", device=dev)
    choice = autotune.tune(batch)
    mats = batch.mats_for(choice.fmt)
    work = batch.workspace()
    plan = fe.fe_cg_batched_plan(mats, batch.b, batch.x, choice.krhs, work,
                                 blocks_per_sm=choice.blocks_per_sm, method=choice.method)
    stream = torch.cuda.Stream(device=dev)
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=stream):
        for x in batch.x:
            x.zero_()
        fe.fe_cg_batched_launch(plan, TOL, MAXIT, stream=stream)
    reps = max(1, min(args.steps, 3))
    graph.replay()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = EV(), EV()
        a.record()
        graph.replay()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    st, res = fe.fe_cg_batched_results(plan)
    t_batched = statistics.mean(ts)
    # the same 64 systems one after another through fe_cg_solve
    xs = [torch.zeros_like(x) for x in batch.x]
    works = {}
    a, b = EV(), EV()
    a.record()
    seq_iters = []
    for i, n in enumerate(sizes):
        A = batch.reps[n].matrix(choice.fmt, "f64")
        if n not in works:
            works[n] = fe.cg_workspace(A, dev)
        r = fe.fe_cg_solve(A.desc, batch.b[i], xs[i], TOL, MAXIT, works[n], check=False)
        seq_iters.append(r.iterations)
    b.record()
    torch.cuda.synchronize()
    t_seq = a.elapsed_time(b)
    diff = max(float(torch.linalg.norm(x - y) / torch.linalg.norm(y)) for x, y in zip(batch.x, xs))
    # untimed: every batched and sequential solution against x* (FP64 CG to
    # 1e-13 on the same system) and the forward-error bound
    # ||x - x*|| <= (||b - A x|| + ||b - A x*||) / lambda_min that any solution
    # meeting the residual test obeys
    rwork = fe.resid_workspace(dev)
    worst = {"batched": 0.0, "sequential": 0.0}
    worst_over_bound = 0.0
    for i, n in enumerate(sizes):
        A = batch.reps[n].matrix(choice.fmt, "f64")
        xst = torch.zeros_like(batch.x[i])
        fe.fe_cg_solve(A.desc, batch.b[i], xst, 1e-13, 20000, works[n], check=False)
        bn = float(torch.linalg.norm(batch.b[i]))
        xsn = float(torch.linalg.norm(xst))
        rs = fe.fe_true_relres(A.desc, batch.b[i], xst, rwork) * bn
        lam = lambda_min_cube(n)
        for key, x in (("batched", batch.x[i]), ("sequential", xs[i])):
            e = float(torch.linalg.norm(x - xst))
            bound = (fe.fe_true_relres(A.desc, batch.b[i], x, rwork) * bn + rs) / lam
            worst[key] = max(worst[key], e / xsn)
            worst_over_bound = max(worst_over_bound, e / bound)
    rows = sum((n + 1) ** 3 for n in sizes)
    nnz = sum((3 * n + 1) ** 3 for n in sizes)
    return {"workload": (f"{len(sizes)} cubic meshes, N ~ U{{32..128}} (PCG64 seed 0), random "
                         f"face data; {rows:,} rows, {nnz:,} stored entries; FP64, one launch"),
            "value": round(t_batched * 1e-3, 6), "unit": "s",
            "sequential_fe_cg_solve_s": round(t_seq * 1e-3, 6),
            "speedup_vs_sequential": round(t_seq / t_batched, 3),
            "status": int(st), "all_converged": all(r.status == 0 for r in res),
            "max_iterations": max(r.iterations for r in res),
            "max_iteration_diff_vs_sequential": max(
                abs(r.iterations - k) for r, k in zip(res, seq_iters)),
            "max_rel_diff_vs_sequential": diff,
            "accuracy": {"max_rel_error_vs_xstar_batched": worst["batched"],
                         "max_rel_error_vs_xstar_sequential": worst["sequential"],
                         "max_error_over_forward_bound": round(worst_over_bound, 4),
                         "all_meet_forward_bound": bool(worst_over_bound <= 1.0),
                         "xstar": "FP64 CG to 1e-13 on each system"},
            "stop_steps": ("two correct runs on these rough-face systems can stop several steps apart: "
                           "on the N=128 system 19 launch shapes of the batched kernel (each its own "
                           "dot-product summation order) stop at 260-277 steps and the oracle at 262; "
                           "the tests hold every system to the residual test, the forward-error bound "
                           "and, for four systems, the oracle's stop step within 20"),
            "distinct_meshes": len(set(sizes)),
            "autotuned": {"format": choice.fmt, "krhs": choice.krhs,
                          "blocks_per_sm": choice.blocks_per_sm,
                          "method": ("single-reduction" if choice.method == fe.BATCH_SINGLE_REDUCTION
                                     else "textbook"),
                          "ms_per_step_probe": round(choice.ms_per_step, 4)},
            "graph_replays_timed": reps}


def exact_minife_faces(n: int):
    """Face array that reproduces the paper's boundary data exactly under the
    face-overwrite order: 1 on the x = 1 face and on the x = 1 edge column of
    every y and z face, 0 elsewhere."""
    import numpy as np
    nn = n + 1
    faces = [np.zeros((nn, nn)) for _ in range(6)]
    faces[1][:, :] = 1.0                 # x1: indexed [iz][iy]
    for k in (2, 3, 4, 5):               # y0, y1 ([iz][ix]); z0, z1 ([iy][ix])
        faces[k][:, n] = 1.0
    return np.concatenate([f.ravel() for f in faces])


if __name__ == "__main__":
    main()
