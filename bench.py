"""Benchmark of the space-time heat BEM hot path on GB300.

One step = one pass of the whole path for every heat capacity constant of
the workload: triangle geometry and pair classification, assembly of all
blocks V^d and K^d, Dirichlet data projection, right-hand side
(1/2 M_h + K_h) g, forward-substitution solve and the L2(Sigma_h) error.
Metric: V,K block entries produced per second (2 E_t E^2 per problem).

Default workload (the large mixed run): icosphere of radius 1 with 5120
triangles, 256 uniform steps on T = 1, alpha = 1, Dirichlet data from 8
seeded exterior heat-kernel sources, FP32 regular pairs and FP32 block
storage (V and K 26.8 GB each).  The headline value is V,K entries per
second of assembly; the whole step's rate, the refined solve, the mixed vs
FP64 comparison on the 3072-triangle cube with 64 steps, the block-Toeplitz
products and the 64-problem batch are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

Under torchrun (N > 1) every rank runs the whole workload on its own GPU
(independent replicas, no collective on the data path; weak scaling).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "V,K entries/s"
UNIT = "entries/s"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 FMA pipe of GB300: 2 FP64 FMA per SM per clock (the nominal 1.25 TFLOP/s
# = 152 SMs x 2 FMA x 2 flop x 2.07 GHz); the regular-pair kernel is bound by it.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP64 flops (DADD + DMUL + 2 DFMA, from ncu's SASS op counters) per
# separated-pair quadrature-point evaluation at one time level i_t >= 1 of
# k_regular_f64, see profiles/.
FP64_FLOPS_PER_EVAL = 137.34
# MUFU (XU) pipe: 32 ex2.approx.f32 per SM per clock (a throughput
# microbenchmark of eight independent ex2 chains per thread measured 9.995e12
# per second = 31.8 per SM per clock at 2.07 GHz on GB300).
MUFU_PEAK_TEX2 = 152 * 32 * 2.07e9 / 1e12


# ncu, k_regular_mixed on the 16-step cube (3072 triangles, alpha 0.5): DRAM
# read 15.19 MB + write 1144.27 MB for 2 x 16 x 3072^2 block entries.
REGULAR_MIXED_DRAM_BYTES_PER_ENTRY = (15.18848e6 + 1144.265e6) / (2 * 16 * 3072.0 ** 2)
# FP64 pipe operations (DFMA, DMUL and DADD, each one slot of the pipe; ncu
# SASS op counters) per evaluation of both potentials -- one point, trial
# triangle, rule point and level -- in k_potential_levels: 1.5509e11
# operations for 1089 x 3072 x 16 x 32 evaluations (profiles/).
POT_FP64_OPS_PER_EVAL = 90.545
# the same for k_regular_nu_f64 (separated pairs, non-uniform grid), per
# quadrature point and positive time difference, the level-0 limits and the
# block updates included: 4.8016e11 operations for 579,896 ordered separated
# pairs x 81 points x 136 differences (768 triangles, geometric 16-step grid;
# profiles/).
NU_FP64_OPS_PER_EVAL = 75.17


def _alu_roofline(kernel, ms, units, unit_name, rate_unit, peak, peak_source, scale=1.0):
    """Roofline record of one launch of an ALU-bound kernel: `units` pipe
    operations (x scale per unit) in `ms` against `peak` (rate_unit)."""
    if not ms:
        return None
    ach = units * scale / (ms / 1e3) / (1e12 if rate_unit.startswith("T") else 1.0)
    return {"kernel": kernel, "launch_ms": ms, "bound": "alu", "unit": rate_unit,
            "achieved": ach, "peak": peak, "frac": ach / peak if peak else None,
            "peak_source": peak_source,
            "units_per_launch": units, "unit_name": unit_name}


def oracle_sample(fn, units, unit, sample):
    """The oracle timed on one host thread for one bounded call fn() that
    computes `units` results: rate in `unit`."""
    t0 = time.perf_counter()
    fn()
    secs = time.perf_counter() - t0
    return {"value": units / secs, "unit": unit, "cores": 1, "kind": "oracle",
            "sample": "%s, %.2f s" % (sample, secs)}


def nu_levels(times):
    """Positive time differences of a grid that the non-uniform assembly
    evaluates (four corners of every block; exact double equality)."""
    t = [float(x) for x in times]
    n = len(t) - 1
    lv = set()
    for k in range(n):
        for i in range(k + 1):
            if i == k:
                lv.add(t[k + 1] - t[k])
            else:
                lv.update((t[k + 1] - t[i + 1], t[k] - t[i + 1], t[k + 1] - t[i], t[k] - t[i]))
    lv.discard(0.0)
    return len(lv)


def mixed_nodes_per_point(n_steps):
    """exp2 evaluations per quadrature point of the mixed separated-pair
    kernel: 6 nodes on interval k = 1 (when n_steps > 2), then chunks of 16
    blocks d0.. whose intervals k = d0..d0+15 (k <= n_steps - 1) take 4, 3 or
    2 nodes (d0 < 16, d0 < 96, otherwise)."""
    if n_steps <= 2:
        return 0
    nodes = 6
    for d0 in range(2, n_steps, 16):
        ng = 4 if d0 < 16 else (3 if d0 < 96 else 2)
        nodes += ng * (min(d0 + 16, n_steps) - d0)
    return nodes


def _measured_hbm_gbs():
    try:
        with open(MEASURED_PEAKS) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0  # fallback figure for a GB300 copy



def _measured_bf16_tflops(sustained=False):
    try:
        with open(MEASURED_PEAKS) as fh:
            d = json.load(fh)
        return float(d["bf16_tflops_sustained" if sustained else "bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1700.0 if sustained else 1900.0  # fallback figures for a GB300


def split_tensor_roofline(E, n, nrhs, ms, sustained=False):
    """Tensor-pipe roofline of one split-operand product (STB_ARITH_SPLIT).
    Algorithmic work: E^2 n (n+1) nrhs flops (each block once per column it
    feeds).  Executed work: 15 bf16 slice products per multiply-add over the
    boxes the kernel runs -- per (tile of 128 rows, box of 64 columns, block d,
    chunk of 64 columns j) 15 x 128 x 64 x 64 multiply-adds, blocks d beyond a
    box's last step skipped -- against the measured dense bf16 peak."""
    rt, nc = -(-E // 128), -(-E // 64)
    mac = 0.0
    for r0 in range(0, nrhs, 64):
        ng = min(64, nrhs - r0)
        rpad = 1
        while rpad < ng:
            rpad *= 2
        S = 64 // rpad
        nblk = sum(min(n, b * S + S) for b in range(-(-n // S)))
        mac += float(rt) * nblk * nc * 15 * 128 * 64 * 64
    peak = _measured_bf16_tflops(sustained)
    exe = 2.0 * mac / (ms / 1e3) / 1e12
    return {"algorithmic_tflops": float(E) * E * n * (n + 1) * nrhs / (ms / 1e3) / 1e12,
            "bf16_slice_tflops_executed": exe, "bf16_peak_tflops": peak,
            "frac_of_bf16_peak": exe / peak,
            "bf16_peak_source": "MEASURED_PEAKS.json %s cuBLAS bf16" % ("sustained" if sustained
                                                                        else "burst")}

HBM_PEAK_GBS = _measured_hbm_gbs()
# FP32 pipe: 128 lanes per SM per clock (one FP32 operation each)
FP32_OP_PEAK = 152 * 128 * 2.07e9


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", default="sphere5120_e256")
    ap.add_argument("--alphas", default=None,
                    help="comma-separated heat capacities (default: the workload's; "
                         "0.5,1,2 for cube3072_e64)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--wave-gb", type=float, default=48.0,
                    help="V+K bytes per memory wave of the batch64 workload")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-potentials", action="store_true",
                    help="skip the potential evaluation report (outside the timed region)")
    ap.add_argument("--serial", action="store_true",
                    help="run the problems of a step one after the other on one stream")
    ap.add_argument("--no-nonuniform", action="store_true",
                    help="skip the non-uniform time grid report (outside the timed region)")
    ap.add_argument("--no-neumann", action="store_true",
                    help="skip the Neumann problem report (outside the timed region)")
    ap.add_argument("--no-p1", action="store_true",
                    help="skip the piecewise-linear data pipeline report (outside the timed region)")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the 64-problem batch report (outside the timed region)")
    ap.add_argument("--no-c3", action="store_true",
                    help="skip the mixed vs FP64 assembly on the icosphere with 5120 triangles and "
                         "128 steps (one FP64 assembly of about 40 s)")
    ap.add_argument("--no-c2", action="store_true",
                    help="skip the reports on the 3072-triangle cube (mixed vs FP64 assembly, the "
                         "three-alpha step) outside the timed region")
    return ap.parse_args()


# heat capacities of a workload when --alphas is not given
WORKLOAD_ALPHAS = {"cube3072_e64": [0.5, 1.0, 2.0]}


def workload_alphas(args, wl):
    if args.alphas:
        return [float(a) for a in args.alphas.split(",")]
    return WORKLOAD_ALPHAS.get(args.workload, [float(wl["alpha"])])


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = []
        with open(self.path) as fh:
            for line in fh:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.remove(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def cpu_oracle_rate(wl, alpha, seconds, threads=1):
    """The FP64 oracle on whole rows of V and K: entries/s.  threads > 1
    runs rows on that many host threads at once (the oracle's C code runs
    with the interpreter lock released), like an OpenMP loop over test
    triangles with dynamic scheduling."""
    import threading
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    E, n = len(wl["tris"]), wl["n_steps"]
    state = {"next": 0, "done": 0}
    lock = threading.Lock()
    t0 = time.perf_counter()

    def worker():
        while time.perf_counter() - t0 < seconds:
            with lock:  # every row once, spread over the mesh
                k = state["next"]
                state["next"] += 1
            if k >= E:
                return
            row = (977 * k) % E
            oracle.assemble_rows(wl["nodes"], wl["tris"], alpha, wl["T"], n, np.array([row]))
            with lock:
                state["done"] += 1

    with ThreadPoolExecutor(max_workers=threads) as ex:
        for f in [ex.submit(worker) for _ in range(threads)]:
            f.result()
    t_used = time.perf_counter() - t0
    return 2.0 * n * E * state["done"] / t_used, state["done"], t_used


def host_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def max_over_ranks(value, world, device):
    """Maximum of a per-rank float over all ranks (the job's time)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step, steps, ms, world):
    """Units of all ranks per second: every rank processes the same work."""
    return world * units_per_rank_step * steps / (ms / 1e3)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    if args.workload == "batch64":
        print(json.dumps({"impl": "reference", "unavailable": "the oracle reference arm times "
                          "single workloads; batch64 is measured on the GPU only"}), flush=True)
        return
    wl = workloads.workload(args.workload)
    alphas = workload_alphas(args, wl)
    E, n = len(wl["tris"]), wl["n_steps"]
    per_step = max(1.0, args.cpu_seconds / 3.0)
    threads = host_threads()
    for i in range(args.warmup):
        cpu_oracle_rate(wl, alphas[i % len(alphas)], per_step / 4, threads)
    rates, rows_total, secs_total = [], 0, 0.0
    for i in range(args.steps):
        r, rows, secs = cpu_oracle_rate(wl, alphas[i % len(alphas)], per_step, threads)
        rates.append(r)
        rows_total += rows
        secs_total += secs
    value = 2.0 * n * E * rows_total / secs_total
    sample = "%d whole rows (all %d blocks of V and K) of %s, alpha cycling %s, %d host threads" % (
        rows_total, n, args.workload, alphas, threads)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * 2 * n * E * E * len(alphas) / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "E": E, "n_steps": n, "alphas": alphas,
                       "quad_regular": 3, "quad_singular": 4},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            # the oracle times whole rows; the step time is the rate scaled to all
            # E rows of every problem of the workload (measured, not scaled, when
            # the sampled rows cover every problem's rows once per timed step)
            "extrapolated": rows_total < E * len(alphas) * args.steps,
            "measured": {"rows": rows_total, "seconds": secs_total, "threads": threads,
                         "entries": 2.0 * n * E * rows_total},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


PEAK_SOURCE = {"fp64": "nominal: 152 SM x 2 FMA/clk x 2 flop x 2.07 GHz",
               "mufu": "nominal: 152 SM x 32 ex2/clk x 2.07 GHz",
               "fp32": "nominal: 152 SM x 128 lanes x 2.07 GHz"}


def measure_pipe_peaks(capi, torch):
    """Replace the nominal FP64 / FP32 / MUFU peaks by the library's probes
    on this device (stb_measure_peaks), and time a cuBLAS TF32 GEMM for
    context; returns the record for the JSON line."""
    global FP64_PEAK_TFLOPS, FP32_OP_PEAK, MUFU_PEAK_TEX2
    f64, f32, ex2 = capi.stb_measure_peaks()
    FP64_PEAK_TFLOPS = 2.0 * f64 / 1e12
    FP32_OP_PEAK = f32
    MUFU_PEAK_TEX2 = ex2 / 1e12
    for k in PEAK_SOURCE:
        PEAK_SOURCE[k] = "measured (stb_measure_peaks: eight independent chains per thread)"
    rec = {"fp64_tflops": FP64_PEAK_TFLOPS, "fp32_fma_per_s": f32, "mufu_tex2_per_s": ex2 / 1e12}
    try:  # TF32 tensor-core reference: cuBLAS SGEMM with TF32 allowed
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = True
        a = torch.randn(8192, 8192, device="cuda")
        c = a @ a
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            c = a @ a
        e1.record()
        torch.cuda.synchronize()
        rec["cublas_tf32_tflops"] = 5 * 2 * 8192.0 ** 3 / (e0.elapsed_time(e1) / 1e3) / 1e12
        torch.backends.cuda.matmul.allow_tf32 = prev
        del a, c
    except RuntimeError:
        rec["cublas_tf32_tflops"] = None
    return rec


def _roofline(name, trace_entry, ms_step, n_reg_pairs, q, n_steps):
    """Roofline of the step's dominant kernel from the live trace (q: points
    per direction of the conical rule, so (q*q)^2 points per pair)."""
    cnt, tot = trace_entry
    launch_ms = tot / cnt
    pts = float(q * q) ** 2
    roof = {"kernel": name, "launch_ms": launch_ms, "share_of_step": tot / ms_step, "traffic": None}
    # the method's own unit, independent of how a kernel evaluates the time
    # integral: one kernel evaluation per separated ordered pair, quadrature
    # point and time level 0..E_t (Sec. 5: each level feeds up to three blocks)
    method = float(n_reg_pairs) * pts * (n_steps + 1)
    roof["method_units"] = {"unit": "kernel evaluations/s", "per_launch": method,
                            "achieved": method / (launch_ms / 1e3),
                            "definition": "separated ordered pairs x points per pair x (E_t + 1) "
                                          "time levels"}
    if name == "k_regular_f64":
        evals = float(n_reg_pairs) * pts * n_steps  # levels 1..E_t
        roof.update({"bound": "alu", "unit": "TFLOP/s", "peak": FP64_PEAK_TFLOPS,
                     "peak_source": "FP64 FMA pipe, " + PEAK_SOURCE["fp64"],
                     "units_per_launch": evals, "unit_name": "separated-pair point-level evaluations"})
        if FP64_FLOPS_PER_EVAL:
            ach = FP64_FLOPS_PER_EVAL * evals / (launch_ms / 1e3) / 1e12
            roof.update({"achieved": ach, "frac": ach / FP64_PEAK_TFLOPS})
    elif name == "k_regular_mixed":
        ex2 = float(n_reg_pairs) * pts * mixed_nodes_per_point(n_steps)
        roof.update({"bound": "alu", "unit": "Tex2/s", "peak": MUFU_PEAK_TEX2,
                     "peak_source": "MUFU ex2 pipe, " + PEAK_SOURCE["mufu"],
                     "units_per_launch": ex2, "unit_name": "MUFU.EX2 time-node evaluations"})
        ach = ex2 / (launch_ms / 1e3) / 1e12
        # DRAM bytes of one launch: ncu capture of this kernel on the 16-step
        # cube (one launch, 2 x 16 x 3072^2 entries), scaled by the entries
        # written (the traffic is the block stores)
        entries = 2.0 * n_steps * float(n_reg_pairs)
        roof.update({"achieved": ach, "frac": ach / MUFU_PEAK_TEX2,
                     "traffic": REGULAR_MIXED_DRAM_BYTES_PER_ENTRY * entries,
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, "
                                       "cube3072_e16 launch scaled by entries written",
                     "algorithmic_bytes": 4.0 * entries})
    else:
        roof.update({"bound": None, "achieved": None, "peak": None, "frac": None})
    return roof


def mixed_vs_fp64_report(capi, pipeline, torch, stream, a_, b_, alpha=0.5, reps_mixed=5,
                         reps_fp64=2, workload="cube3072_e64", fp64_warmup=True):
    """Mixed-precision against FP64 assembly of V and K (by default on the cube
    with 3072 triangles and 64 steps): CUDA events around the whole
    stb_assemble call (geometry, pair classification, rule tables and
    kernels) for both, one warm-up call each (for FP64 optional: a long call
    needs none once the kernels have run), the median of the timed calls;
    relative Frobenius error of every mixed block against the FP64 block; then
    the other stages of the mixed problem (projection, right-hand side,
    refined solve, error)."""
    wl = workloads.workload(workload)
    nodes, tris, n, src = wl["nodes"], wl["tris"], wl["n_steps"], wl["sources"]
    mesh = capi.Mesh(nodes, tris)
    E = len(tris)
    pm = pipeline.DirichletProblem(nodes, tris, alpha, wl["T"], n, src, mesh=mesh,
                                   precision=capi.STB_PREC_MIXED, storage=capi.STB_STORE_F32)
    pf = pipeline.DirichletProblem(nodes, tris, alpha, wl["T"], n, src, mesh=mesh)

    def timed(fn, reps, warm=True):
        if warm:
            fn(stream)
            torch.cuda.synchronize()
        out = []
        for _ in range(reps):
            a_.record(stream)
            fn(stream)
            b_.record(stream)
            torch.cuda.synchronize()
            out.append(a_.elapsed_time(b_))
        return out

    tm = timed(pm.assemble, reps_mixed)
    tf = timed(pf.assemble, reps_fp64, fp64_warmup)
    errs = {}
    for name, A, B in (("V", pm.V, pf.V), ("K", pm.K, pf.K)):
        errs[name] = max(float(torch.linalg.norm(A[d].double() - B[d]) / torch.linalg.norm(B[d]))
                         for d in range(n))
    del pf
    torch.cuda.empty_cache()
    entries = 2.0 * n * E * E
    mm, mf = statistics.median(tm), statistics.median(tf)
    stages = {"assemble": mm}
    for label, fn in (("project", pm.project), ("rhs", pm.rhs), ("solve", pm.solve),
                      ("error", pm.error)):
        stages[label] = statistics.median(timed(fn, 2))
    refinements, rel_residual = capi.stb_solve_report(pm.ws_solve)
    out = {"workload": workload, "alpha": alpha, "entries": entries,
           "timing": "CUDA events around the whole stb_assemble call, one warm-up call (FP64: %s), "
                     "median of the timed calls" % ("yes" if fp64_warmup else
                                                    "none, the kernels ran in the report before"),
           "fp64_assembly_ms": mf, "fp64_runs_ms": tf, "fp64_entries_per_s": entries / (mf / 1e3),
           "mixed_assembly_ms": mm, "mixed_runs_ms": tm, "mixed_entries_per_s": entries / (mm / 1e3),
           "speedup": mf / mm, "max_block_rel_err_mixed_vs_fp64": errs,
           "stated_bound_per_block": 2e-6,
           "mixed_problem_stage_ms": stages, "mixed_solve_refinements": refinements,
           "mixed_solve_rel_residual": rel_residual, "rel_l2_error_w": pm.relative_error()}
    del pm
    torch.cuda.empty_cache()
    return out


def nonuniform_report(capi, pipeline, torch, stream, a_, b_, cpu=True):
    """FP64 Dirichlet problem on a geometric time grid (ratio 1.2, 16 steps,
    T = 1) and on the uniform grid of the same step count: assembly and
    solve times, relative L2 errors of w_h (source (1.5,1.5,1.5), t0 = 0);
    the roofline of the separated-pair kernel on the geometric grid and the
    oracle's rows of the same blocks."""
    nodes, tris = workloads.cube_mesh(8)
    src = workloads.point_source((1.5, 1.5, 1.5), t0=0.0)
    n, ratio = 16, 1.2
    steps = ratio ** np.arange(n)
    times = np.concatenate([[0.0], np.cumsum(steps / steps.sum())])
    times[-1] = 1.0
    E = len(tris)
    out = {"workload": "cube, 768 triangles, 16 steps, T = 1, alpha 1",
           "grid": "geometric, ratio %.1f" % ratio}
    for label, t in (("geometric", times), ("uniform", np.arange(n + 1) / n)):
        pr = pipeline.NonUniformDirichletProblem(nodes, tris, 1.0, t, src)
        pr.run(stream)
        torch.cuda.synchronize()
        capi.stb_trace_enable(True)
        capi.stb_trace_reset()
        a_.record(stream)
        capi.stb_assemble_nu(pr.mesh, pr.params, pr.times, pr.V, pr.K, pr.ws_assemble, stream)
        b_.record(stream)
        torch.cuda.synchronize()
        capi.stb_trace_enable(False)
        tr = capi.stb_trace_read()
        asm_ms = a_.elapsed_time(b_)
        a_.record(stream)
        capi.stb_solve_nu(pr.V, pr.E, pr.n_steps, pr.nrhs, pr.f, pr.w, pr.ws_solve, stream)
        b_.record(stream)
        torch.cuda.synchronize()
        n_blocks = n * (n + 1) // 2
        out[label] = {"assembly_ms": asm_ms, "solve_ms": a_.elapsed_time(b_),
                      "rel_l2_error_w": pr.relative_error(), "distinct_levels": nu_levels(t),
                      "entries_per_s": 2.0 * n_blocks * E * E / (asm_ms / 1e3),
                      "kernels_ms": {k: v[1] for k, v in tr.items()}}
        if label == "geometric":
            n_reg = E * E - 2 * pr.mesh.n_touching + E
            evals = float(n_reg) * 81.0 * nu_levels(t)
            reg_ms = tr.get("k_regular_nu_f64", (1, 0.0))[1]
            if NU_FP64_OPS_PER_EVAL:
                out["roofline"] = _alu_roofline(
                    "k_regular_nu_f64", reg_ms, evals,
                    "separated-pair point-level evaluations x FP64 operations per evaluation (ncu)",
                    "FP64 op/s", FP64_PEAK_TFLOPS * 1e12 / 2, "FP64 pipe, " + PEAK_SOURCE["fp64"],
                    scale=NU_FP64_OPS_PER_EVAL)
            else:
                out["point_level_evals_per_s"] = evals / (reg_ms / 1e3) if reg_ms else None
            if cpu:
                import oracle
                rows = np.array([0, E // 2])
                out["cpu_baseline"] = oracle_sample(
                    lambda: oracle.assemble_rows_nu(nodes, tris, 1.0, t, rows), 2.0 * n_blocks * E * 2,
                    "entries/s", "2 whole rows (all 136 blocks of V and K) of the geometric grid")
            # the same grid with the separated pairs in FP32: times, block
            # errors against the FP64 blocks above, solution and error
            pm = pipeline.NonUniformDirichletProblem(nodes, tris, 1.0, t, src,
                                                     precision=capi.STB_PREC_MIXED)
            pm.run(stream)
            torch.cuda.synchronize()
            capi.stb_trace_enable(True)
            capi.stb_trace_reset()
            a_.record(stream)
            capi.stb_assemble_nu(pm.mesh, pm.params, pm.times, pm.V, pm.K, pm.ws_assemble, stream)
            b_.record(stream)
            torch.cuda.synchronize()
            capi.stb_trace_enable(False)
            trm = capi.stb_trace_read()
            m_ms = a_.elapsed_time(b_)
            ev = ((pm.V - pr.V).flatten(1).norm(dim=1) / pr.V.flatten(1).norm(dim=1)).max()
            ek = ((pm.K - pr.K).flatten(1).norm(dim=1) / pr.K.flatten(1).norm(dim=1)).max()
            cf_terms, g_nodes, _ = capi.stb_assemble_nu_mixed_counts(pm.params, t)
            reg_m = trm.get("k_regular_nu_mixed", (1, 0.0))[1]
            roof_m = _alu_roofline(
                "k_regular_nu_mixed", reg_m, float(n_reg) * 81.0 * g_nodes,
                "MUFU.EX2 Gauss-node evaluations (the %d closed-form evaluations per point, "
                "erfc and exp each, not counted)" % cf_terms, "Tex2/s", MUFU_PEAK_TEX2,
                "MUFU ex2 pipe, " + PEAK_SOURCE["mufu"])
            out["geometric_mixed"] = {
                "roofline": roof_m, "gauss_nodes": g_nodes, "closed_form_evaluations": cf_terms,
                "assembly_ms": m_ms, "entries_per_s": 2.0 * n_blocks * E * E / (m_ms / 1e3),
                "speedup_vs_fp64": asm_ms / m_ms,
                "max_block_rel_err_vs_fp64": {"V": float(ev), "K": float(ek)},
                "rel_l2_error_w": pm.relative_error(),
                "rel_diff_w_vs_fp64": float((pm.w - pr.w).norm() / pr.w.norm()),
                "kernels_ms": {k: v[1] for k, v in trm.items()}}
            del pm
        del pr
    return out


def potentials_report(capi, stream, a_, b_, cpu=True):
    """Times of the single- plus double-layer potential at the 34848 points
    of the potential benchmark: per-point kernel and the level-block form;
    the roofline of the level kernel and the oracle at the latest points."""
    import torch
    nodes, tris = workloads.cube_mesh(16, lo=-1.0, hi=1.0)
    T, n, alpha = 1.0, 32, 0.5
    mesh = capi.Mesh(nodes, tris)
    prm = capi.stb_default_params(alpha, T, n)
    pts = workloads.reprsc_points(n, T)
    P = len(pts) // n
    rng = np.random.default_rng(1089)
    w_h = rng.normal(size=(1, n, len(tris)))
    u1_h = rng.normal(size=(1, n, len(nodes)))
    w = torch.tensor(w_h, device="cuda")
    u1 = torch.tensor(u1_h, device="cuda")
    out = {"workload": "cube (-1,1)^3, 3072 triangles, 32 steps, 1089 points x 32 step midpoints",
           "q_space": 4}
    pts_d = torch.tensor(pts, device="cuda")
    s1 = torch.empty((1, len(pts)), dtype=torch.float64, device="cuda")
    d1 = torch.empty_like(s1)
    ws = torch.empty(capi.stb_potentials_workspace_size(mesh, prm, 1, len(pts), 4),
                     dtype=torch.uint8, device="cuda")
    capi.stb_potentials(mesh, prm, pts_d, w, u1, 1, s1, d1, ws)
    a_.record(stream)
    capi.stb_potentials(mesh, prm, pts_d, w, u1, 1, s1, d1, ws)
    b_.record(stream)
    torch.cuda.synchronize()
    out["per_point_ms"] = a_.elapsed_time(b_)
    # the per-point kernel with FP32 level values
    prm_pm = capi.stb_default_params(alpha, T, n, precision=capi.STB_PREC_MIXED)
    s1m, d1m = torch.empty_like(s1), torch.empty_like(d1)
    capi.stb_potentials(mesh, prm_pm, pts_d, w, u1, 1, s1m, d1m, ws)
    a_.record(stream)
    capi.stb_potentials(mesh, prm_pm, pts_d, w, u1, 1, s1m, d1m, ws)
    b_.record(stream)
    torch.cuda.synchronize()
    out["per_point_mixed"] = {
        "ms": a_.elapsed_time(b_),
        "max_rel_diff_vs_fp64": float(max((s1m - s1).abs().max() / s1.abs().max(),
                                          (d1m - d1).abs().max() / d1.abs().max()))}
    del ws
    p3 = torch.tensor(pts[:P, :3], device="cuda")
    s2 = torch.empty((1, n, P), dtype=torch.float64, device="cuda")
    d2 = torch.empty_like(s2)
    ws = torch.empty(capi.stb_potentials_grid_workspace_size(mesh, prm, 1, P, 4),
                     dtype=torch.uint8, device="cuda")
    eps = 0.5 * T / n
    capi.stb_potentials_grid(mesh, prm, p3, eps, w, u1, 1, s2, d2, ws)
    torch.cuda.synchronize()
    capi.stb_trace_enable(True)
    capi.stb_trace_reset()
    a_.record(stream)
    capi.stb_potentials_grid(mesh, prm, p3, eps, w, u1, 1, s2, d2, ws)
    b_.record(stream)
    torch.cuda.synchronize()
    capi.stb_trace_enable(False)
    tr = capi.stb_trace_read()
    out["level_blocks_ms"] = a_.elapsed_time(b_)
    out["kernels_ms"] = {k: v[1] for k, v in tr.items()}
    out["max_rel_diff_between_forms"] = float(max(
        (s2.reshape(1, -1) - s1).abs().max() / s1.abs().max(),
        (d2.reshape(1, -1) - d1).abs().max() / d1.abs().max()))
    evals = float(P) * len(tris) * 16 * n
    out["level_evaluations_per_s"] = evals / (out["level_blocks_ms"] / 1e3)
    out["roofline"] = _alu_roofline(
        "k_potential_levels", tr.get("k_potential_levels", (1, 0.0))[1], evals,
        "point-triangle-rule point-level evaluations of both potentials x FP64 operations per "
        "evaluation (ncu)", "FP64 op/s", FP64_PEAK_TFLOPS * 1e12 / 2,
        "FP64 pipe, " + PEAK_SOURCE["fp64"], scale=POT_FP64_OPS_PER_EVAL)
    # the level blocks from FP32 quadrature points
    prm_m = capi.stb_default_params(alpha, T, n, precision=capi.STB_PREC_MIXED)
    s3 = torch.empty_like(s2)
    d3 = torch.empty_like(d2)
    capi.stb_potentials_grid(mesh, prm_m, p3, eps, w, u1, 1, s3, d3, ws)
    torch.cuda.synchronize()
    capi.stb_trace_enable(True)
    capi.stb_trace_reset()
    a_.record(stream)
    capi.stb_potentials_grid(mesh, prm_m, p3, eps, w, u1, 1, s3, d3, ws)
    b_.record(stream)
    torch.cuda.synchronize()
    capi.stb_trace_enable(False)
    trm = capi.stb_trace_read()
    out["level_blocks_mixed"] = {
        "ms": a_.elapsed_time(b_), "kernels_ms": {k: v[1] for k, v in trm.items()},
        "max_rel_diff_vs_fp64": float(max((s3 - s2).abs().max() / s2.abs().max(),
                                          (d3 - d2).abs().max() / d2.abs().max()))}
    out["paper_36_threads_s"] = {"single_layer": 0.31, "double_layer": 0.82,
                                 "note": "Table reprsc, 2 x 18-core Xeon Gold 6240; context"}
    del ws
    if cpu:  # the oracle at the 4 latest points (all 32 levels each)
        import oracle
        sel = pts[-4:]
        out["cpu_baseline"] = oracle_sample(
            lambda: oracle.potentials(nodes, tris, alpha, T, n, sel, w=w_h, u1=u1_h, q=4),
            4.0 * len(tris) * 16 * n, "evaluations/s",
            "both potentials at the 4 points of the last step midpoint (32 levels each)")
    return out


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2102_09811_gb300 import capi, pipeline

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    wl = workloads.workload(args.workload)
    alphas = workload_alphas(args, wl)
    E, n = len(wl["tris"]), wl["n_steps"]
    nodes, tris, src = wl["nodes"], wl["tris"], wl["sources"]
    mixed = args.precision == "mixed"
    prec = capi.STB_PREC_MIXED if mixed else capi.STB_PREC_FP64
    storage = capi.STB_STORE_F32 if mixed else capi.STB_STORE_F64
    pipe_peaks = measure_pipe_peaks(capi, torch)
    mesh = capi.Mesh(nodes, tris)
    probs = [pipeline.DirichletProblem(nodes, tris, a, wl["T"], n, src, mesh=mesh, precision=prec,
                                       storage=storage) for a in alphas]
    stream = torch.cuda.current_stream()
    # one stream per problem: the problems are independent, so the latency-
    # bound phases of one (the march, the factorisation) overlap the compute-
    # bound assembly of another (set up after the synchronous warm-up)
    streams = [stream] * len(probs)

    trace_assembly = [False]  # trace the first problem's assembly kernels only
    # CUDA events around every assembly of the timed steps: the metric's time
    # (V,K entries per second of assembly, one list entry per step)
    asm_events = []

    def run_problem(i, p, s, after=None):
        if after is not None:  # the previous problem's assembly
            s.wait_event(after)
        a0 = torch.cuda.Event(enable_timing=True)
        a0.record(s)
        if i == 0 and trace_assembly[0]:
            capi.stb_trace_enable(True)
            p.assemble(s)
            capi.stb_trace_enable(False)
        else:
            p.assemble(s)
        done = torch.cuda.Event(enable_timing=True)
        done.record(s)
        if asm_events:
            asm_events[-1].append((a0, done))
        p.project(s)
        p.rhs(s)
        p.solve(s)
        p.error(s)
        return done

    def step():
        if streams[0] is stream:
            for i, p in enumerate(probs):
                run_problem(i, p, stream)
            return
        # the assemblies (compute-bound, each filling the GPU) run one after
        # the other; each problem's data, right-hand side, solve and error
        # (latency-bound phases) overlap the next problem's assembly
        ev = torch.cuda.Event()
        ev.record(stream)
        prev = None
        for i, (p, s) in enumerate(zip(probs, streams)):
            s.wait_event(ev)
            prev = run_problem(i, p, s, prev)
        for s in streams:
            e = torch.cuda.Event()
            e.record(s)
            stream.wait_event(e)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    concurrent = not args.serial and len(probs) > 1
    if concurrent and args.warmup == 0:  # a synchronous pass gives the refinement counts
        step()
        barrier()
    if concurrent:  # refinement counts of the synchronous warm-up solves
        for p in probs:
            p.set_async(p.solve_status()[0])
        streams[:] = [torch.cuda.Stream() for _ in probs]
    # the timed steps trace (CUDA events around each launch) the assembly of
    # the first problem only: the dominant kernel's live launch times at
    # negligible cost (tracing every launch slows the host-bound march)
    trace_assembly[0] = True
    step()
    barrier()
    capi.stb_trace_reset()
    capi.stb_trace_reset()
    launches0 = capi.stb_launch_count()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        barrier()
        start.record(stream)
        for _ in range(args.steps):
            asm_events.append([])
            step()
        end.record(stream)
        barrier()
    capi.stb_trace_enable(False)
    launches = capi.stb_launch_count() - launches0
    trace = capi.stb_trace_read()
    ms = max_over_ranks(start.elapsed_time(end), world, "cuda")
    entries = 2.0 * n * E * E * len(alphas)
    # the metric: entries per second of assembly (CUDA events around every
    # problem's assembly; the best timed step, the slowest rank), and the
    # whole step's rate beside it
    asm_ms_steps = [sum(a.elapsed_time(b) for a, b in ev) for ev in asm_events]
    asm_ms_best = max_over_ranks(min(asm_ms_steps), world, "cuda")
    asm_ms_mean = max_over_ranks(statistics.mean(asm_ms_steps), world, "cuda")
    value = world * entries / (asm_ms_best / 1e3)
    step_rate = whole_job_rate(entries, args.steps, ms, world)
    rel_err = [p.relative_error() for p in probs]
    solve_status = [p.solve_status() for p in probs]
    if any(st != 0 for _, _, st in solve_status):
        raise RuntimeError("a solve of the timed steps did not converge: %s" % solve_status)
    n_reg_pairs = E * E - 2 * mesh.n_touching + E  # ordered separated pairs
    name = "k_regular_mixed" if mixed else "k_regular_f64"
    # share of the step: the traced (first) problem's launches stand for all
    roof = _roofline(name, trace[name], ms / len(probs), n_reg_pairs, 3, n)
    roof["traced_launches"] = "the first problem's assembly, every timed step"

    # block-Toeplitz matvec on the assembled V of the first problem, in each
    # arithmetic the stored blocks allow; errors relative to the FP64 product
    p0 = probs[0]
    y = torch.empty_like(p0.w)
    # the SIMT FP64 and double-float forms take seconds at 8 right-hand sides x
    # 5120^2 x 256 steps: they run only up to the 3072 x 64 size
    small = float(E) * E * n * (n + 1) * p0.nrhs <= 1e11
    ariths = [("fp64", capi.STB_ARITH_FP64)] if small or storage == capi.STB_STORE_F64 else []
    if storage == capi.STB_STORE_F32:
        ariths = [("split", capi.STB_ARITH_SPLIT)] + ariths
        if small:
            ariths += [("df", capi.STB_ARITH_DF)]
        ariths += [("tf32", capi.STB_ARITH_TF32)]
    a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flops = float(E) * E * n * (n + 1) * p0.nrhs
    a_bytes = float(n) * E * E * (4 if storage == capi.STB_STORE_F32 else 8)
    matvec, y_ref = {}, None
    for label, ar in ariths:
        ws = torch.empty(capi.stb_toeplitz_ex_workspace_size(E, n, p0.nrhs, ar), dtype=torch.uint8,
                         device="cuda")
        capi.stb_toeplitz_matvec_ex(p0.V, storage, E, n, p0.nrhs, p0.w, 0.0, y, ar, ws)
        capi.stb_workspace_status(ws)
        if y_ref is None:
            y_ref = y.clone()
        rel = float(torch.linalg.norm(y - y_ref) / torch.linalg.norm(y_ref))
        reps = 5 if label == "fp64" else (20 if small else 3)
        a_.record(stream)
        for _ in range(reps):
            capi.stb_toeplitz_matvec_ex(p0.V, storage, E, n, p0.nrhs, p0.w, 0.0, y, ar, ws)
        b_.record(stream)
        torch.cuda.synchronize()
        mv_ms = a_.elapsed_time(b_) / reps
        macs = flops / 2.0
        entry = {"ms": mv_ms, "tflops": flops / (mv_ms / 1e3) / 1e12,
                 "block_gbs": a_bytes / (mv_ms / 1e3) / 1e9,
                 "rel_err_vs_" + ariths[0][0]: rel}
        if label == "fp64":  # FP64 FMA pipe, one DFMA per multiply-add
            entry["frac_of_fp64_fma_peak"] = macs / (mv_ms / 1e3) / (FP64_PEAK_TFLOPS * 1e12 / 2)
        elif label == "df":  # FP32 pipe, 11 FP32 operations per multiply-add
            entry["frac_of_fp32_op_peak"] = 11.0 * macs / (mv_ms / 1e3) / FP32_OP_PEAK
        elif label == "split":  # 15 bf16 slice products per multiply-add on the tensor cores
            entry.update(split_tensor_roofline(E, n, p0.nrhs, mv_ms))
        else:  # HBM: every block read once
            entry["frac_of_hbm_peak"] = a_bytes / (mv_ms / 1e3) / 1e9 / HBM_PEAK_GBS
        matvec[label] = entry
        del ws
    best = "split" if "split" in matvec else "fp64"
    mv_tflops, mv_ms = matvec[best]["tflops"], matvec[best]["ms"]
    matvec["blocks_read_gb"] = a_bytes / 1e9
    matvec["hbm_peak_gbs"] = HBM_PEAK_GBS

    # stage times of one problem (CUDA events, outside the timed region) and
    # the refinement report of its solve
    stage_ms = {}
    capi.stb_trace_reset()
    capi.stb_trace_enable(True)
    for label, fn in (("assemble", p0.assemble), ("project", p0.project), ("rhs", p0.rhs),
                      ("solve", p0.solve), ("error", p0.error)):
        a_.record(stream)
        fn(stream)
        b_.record(stream)
        torch.cuda.synchronize()
        stage_ms[label] = a_.elapsed_time(b_)
    capi.stb_trace_enable(False)
    one = capi.stb_trace_read()
    refinements, rel_residual = capi.stb_solve_report(p0.ws_solve)
    solve_info = {"stage_ms": stage_ms, "refinements": refinements, "rel_residual": rel_residual,
                  "alpha": alphas[0], "kernels_ms_one_problem": {k: v[1] for k, v in one.items()}}
    # rooflines of the solve's tensor-core kernels from the same trace: the
    # split-operand product (right-hand side and refinement residuals) and the
    # march's far history (HBM: the blocks each panel reads)
    if "k_toeplitz_split" in one:
        cnt, tot = one["k_toeplitz_split"]
        solve_info["roofline_split_product"] = dict(
            kernel="k_toeplitz_split", launches=cnt, launch_ms=tot / cnt, bound="tensor",
            **split_tensor_roofline(E, n, p0.nrhs, tot / cnt, sustained=True))
    if "k_toeplitz_panel" in one:
        cnt, tot = one["k_toeplitz_panel"]
        per_march = sum((kp + min(8, n - kp) - 1) for kp in range(8, n, 8)) * 4.0 * E * E
        marches = cnt / max(1, len(range(8, n, 8)))
        ach = per_march * marches / (tot / 1e3) / 1e9
        solve_info["roofline_far_history"] = {
            "kernel": "k_toeplitz_panel", "launches": cnt, "launch_ms": tot / cnt, "bound": "hbm",
            "unit": "GB/s", "achieved": ach, "peak": HBM_PEAK_GBS, "frac": ach / HBM_PEAK_GBS,
            "algorithmic_bytes_per_march": per_march,
            "note": "blocks 1 .. kp+7 of V read once per panel of 8 steps (FP32)"}

    # the other precision on the 3072-triangle cube with 64 steps (the FP64 GPU
    # baseline workload): both assemblies timed alike, per-block errors
    cmp = cmp3 = None
    if mixed and not args.no_fp64_compare and not args.no_c2:
        cmp = mixed_vs_fp64_report(capi, pipeline, torch, stream, a_, b_)
    # the same on the precision workload (icosphere 5120, 128 steps, alpha 1):
    # one FP64 assembly of about 40 s (its kernels are warm from the cube)
    if mixed and not args.no_fp64_compare and not args.no_c3:
        cmp3 = mixed_vs_fp64_report(capi, pipeline, torch, stream, a_, b_, alpha=1.0,
                                    reps_mixed=3, reps_fp64=1, workload="sphere5120_e128",
                                    fp64_warmup=args.no_c2)

    # V and the right-hand side without storing K (matrix-free K g), first
    # problem: time against assembly + stored-K right-hand side
    mfree = None
    if mixed and p0.nrhs * n <= 128:
        f_mf = torch.empty_like(p0.f)
        ws_mf = torch.empty(capi.stb_assemble_vrhs_workspace_size(mesh, p0.params, p0.nrhs),
                            dtype=torch.uint8, device="cuda")
        capi.stb_assemble_vrhs(mesh, p0.params, p0.V, p0.g, p0.nrhs, f_mf, ws_mf, stream)
        torch.cuda.synchronize()
        a_.record(stream)
        capi.stb_assemble_vrhs(mesh, p0.params, p0.V, p0.g, p0.nrhs, f_mf, ws_mf, stream)
        b_.record(stream)
        torch.cuda.synchronize()
        mf_ms = a_.elapsed_time(b_)
        p0.assemble(stream)
        p0.rhs(stream)
        torch.cuda.synchronize()
        mfree = {"ms": mf_ms, "stored_path_ms": stage_ms["assemble"] + stage_ms["rhs"],
                 "rel_diff_f": float((torch.linalg.norm(f_mf - p0.f) / torch.linalg.norm(p0.f))),
                 "k_bytes_not_stored": 4.0 * n * E * E}
        del ws_mf, f_mf

    # the extension reports below run on the 3072-triangle cube with 64 steps
    # (the paper's scalability mesh), whatever the headline workload
    wlx = workloads.workload("cube3072_e64")
    nodes_x, tris_x, n_x, src_x = wlx["nodes"], wlx["tris"], wlx["n_steps"], wlx["sources"]
    mesh_x = capi.Mesh(nodes_x, tris_x)
    E_x = len(tris_x)
    n_reg_pairs_x = E_x * E_x - 2 * mesh_x.n_touching + E_x
    alpha_x = 0.5
    # the paper's own discretisation of the data (piecewise-linear in space,
    # Sec. 3.2 / 3.4) for the first problem: stage times after one warm-up
    # pass, the K1 kernels' share and the point-level evaluation rate
    p1 = None
    if not args.no_p1:
        pp = pipeline.DirichletProblem(nodes_x, tris_x, alpha_x, wlx["T"], n_x, src_x, mesh=mesh_x,
                                       precision=prec, storage=storage, data="p1")
        pp.run(stream)
        torch.cuda.synchronize()
        capi.stb_trace_enable(True)
        capi.stb_trace_reset()
        p1_ms = {}
        for label, fn in (("assemble", pp.assemble), ("project", pp.project), ("rhs", pp.rhs),
                          ("solve", pp.solve), ("error", pp.error)):
            a_.record(stream)
            fn(stream)
            b_.record(stream)
            torch.cuda.synchronize()
            p1_ms[label] = a_.elapsed_time(b_)
        capi.stb_trace_enable(False)
        tr1 = capi.stb_trace_read()
        kind = "mixed" if "k_regular_k1_mixed" in tr1 else "f64"
        k1_ms = tr1.get("k_regular_k1_" + kind, (1, 0.0))[1]
        p1 = {"alpha": alpha_x, "workload": "cube3072_e64", "stage_ms": p1_ms, "rel_l2_error_w": pp.relative_error(),
              "k1_arithmetic": kind, "k_regular_k1_ms": k1_ms,
              "k_singular_k1_ms": tr1.get("k_singular_k1_" + kind, (1, 0.0))[1],
              "k1_entries": float(n_x) * E_x * mesh_x.n_nodes,
              "kernels_ms": {k: v[1] for k, v in tr1.items()}}
        k1_all = k1_ms + p1["k_singular_k1_ms"]
        p1["k1_entries_per_s"] = p1["k1_entries"] / (k1_all / 1e3) if k1_all else None
        if kind == "mixed":  # one exp2 per node and point, as for V, K
            p1["roofline"] = _alu_roofline(
                "k_regular_k1_mixed", k1_ms, float(n_reg_pairs_x) * 81.0 * mixed_nodes_per_point(n_x),
                "MUFU.EX2 time-node evaluations", "Tex2/s", MUFU_PEAK_TEX2,
                "MUFU ex2 pipe, " + PEAK_SOURCE["mufu"])
        elif k1_ms:
            p1["roofline"] = _alu_roofline(
                "k_regular_k1_f64", k1_ms, float(n_reg_pairs_x) * 81.0 * n_x,
                "separated-pair point-level evaluations", "point-level evaluations/s", None, None)
        if not args.no_cpu_baseline:  # the oracle's K1 on whole test-triangle rows
            import oracle
            rows = np.array([0, E_x // 2])
            p1["cpu_baseline"] = oracle_sample(
                lambda: oracle.assemble_k1_rows(nodes_x, tris_x, alpha_x, wlx["T"], n_x, rows),
                2.0 * n_x * mesh_x.n_nodes, "K1 entries/s",
                "2 whole rows of K1 (all %d blocks x %d nodes) of %s" % (n_x, mesh_x.n_nodes,
                                                                      "cube3072_e64"))
        del pp

    # the Neumann problem (Sec. 3.3) on the same cube:
    # stage times after a warm-up pass, the hypersingular kernels' times
    neu = None
    if not args.no_neumann:
        pn = pipeline.NeumannProblem(nodes_x, tris_x, alpha_x, wlx["T"], n_x, src_x, mesh=mesh_x,
                                     precision=prec, storage=storage)
        pn.run(stream)
        torch.cuda.synchronize()
        capi.stb_trace_enable(True)
        capi.stb_trace_reset()
        nms = {}
        for label, fn in (("assemble", pn.assemble), ("project", pn.project), ("rhs", pn.rhs),
                          ("solve", pn.solve), ("error", pn.error)):
            a_.record(stream)
            fn(stream)
            b_.record(stream)
            torch.cuda.synchronize()
            nms[label] = a_.elapsed_time(b_)
        capi.stb_trace_enable(False)
        trn = capi.stb_trace_read()
        neu = {"alpha": alpha_x, "workload": "cube3072_e64", "stage_ms": nms, "rel_l2_error_u": pn.relative_error(),
               "kernels_ms": {k: v[1] for k, v in trn.items()}}
        d2k = "mixed" if "k_regular_d2_mixed" in trn else "f64"
        d2_ms = trn.get("k_regular_d2_" + d2k, (1, 0.0))[1]
        d2_all = d2_ms + trn.get("k_singular_d2_" + d2k, (1, 0.0))[1]
        neu["d2_pair_blocks_per_s"] = float(E_x) * E_x * n_x / (d2_all / 1e3) if d2_all else None
        if d2k == "mixed":  # one exp2 per node and point, as for V, K
            neu["roofline"] = _alu_roofline(
                "k_regular_d2_mixed", d2_ms, float(n_reg_pairs_x) * 81.0 * mixed_nodes_per_point(n_x),
                "MUFU.EX2 time-node evaluations", "Tex2/s", MUFU_PEAK_TEX2,
                "MUFU ex2 pipe, " + PEAK_SOURCE["mufu"])
        # D^1: one FP64 FMA per star pair and block, (sum of star sizes)^2 =
        # (3 E)^2 per block
        neu["roofline_d1"] = _alu_roofline(
            "k_hypersingular_d1", trn.get("k_hypersingular_d1", (1, 0.0))[1],
            9.0 * E_x * E_x * n_x, "FP64 FMA (one per star pair and block)", "FMA/s",
            FP64_PEAK_TFLOPS * 1e12 / 2, "FP64 pipe, " + PEAK_SOURCE["fp64"])
        if not args.no_cpu_baseline:  # the oracle's D^2 on whole test-triangle rows
            import oracle
            rows = np.array([0, E_x // 3, E_x // 2])
            neu["cpu_baseline"] = oracle_sample(
                lambda: oracle.assemble_d2(nodes_x, tris_x, alpha_x, wlx["T"], n_x, test_tris=rows),
                3.0 * E_x * n_x, "triangle-pair blocks/s",
                "D^2 of 3 test triangles (all %d trial triangles and %d blocks) of %s"
                % (E_x, n_x, "cube3072_e64"))
        del pn
        torch.cuda.empty_cache()

    # a non-uniform (geometric) time grid against the uniform one, FP64, on a
    # cube of 768 triangles with 16 steps: times, the number of distinct time
    # differences and the errors
    nonuni = None
    if not args.no_nonuniform:
        nonuni = nonuniform_report(capi, pipeline, torch, stream, a_, b_,
                                   cpu=not args.no_cpu_baseline)

    # the representation formula's potentials on the workload of the paper's
    # potential benchmark (Table reprsc: cube (-1,1)^3, 3072 triangles, 32
    # steps, 33 x 33 points x 32 step midpoints = 34848 points), seeded
    # densities; both kernels, FP64
    pots = None
    if not args.no_potentials:
        pots = potentials_report(capi, stream, a_, b_, cpu=not args.no_cpu_baseline)

    # end to end through the public API from host buffers (mesh, sources in;
    # solution and error norms out)
    e2e = None
    if not args.no_e2e:
        h2d = d2h = 0
        n_e2e = max(1, min(args.steps, 2))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            prs, outs = [], []
            for i, a in enumerate(alphas):
                pr = pipeline.DirichletProblem(nodes, tris, a, wl["T"], n, src, precision=prec,
                                               storage=storage)
                s_i = streams[i]
                if concurrent:  # the refinement count of the timed problems
                    pr.set_async(probs[i].solve_status()[0])
                    s_i.wait_stream(stream)
                pr.run(s_i)
                with torch.cuda.stream(s_i):
                    w_host = torch.empty(pr.w.shape, dtype=pr.w.dtype, pin_memory=True)
                    err_host = torch.empty(pr.err.shape, dtype=pr.err.dtype, pin_memory=True)
                    w_host.copy_(pr.w, non_blocking=True)
                    err_host.copy_(pr.err, non_blocking=True)
                prs.append(pr)
                outs.append((w_host, err_host))
                h2d += nodes.nbytes + tris.nbytes + src.nbytes
                d2h += w_host.numel() * 8 + err_host.numel() * 8
            torch.cuda.synchronize()
            if concurrent:
                assert all(pr.solve_status()[2] == 0 for pr in prs), "an asynchronous solve failed"
            del prs, outs
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e = {"value": world * entries * n_e2e / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": h2d // n_e2e, "d2h_bytes_per_step": d2h // n_e2e}

    # the 64-problem batch of ellipsoids (its own report, outside the timed region)
    batch = None
    if mixed and not args.no_batch:
        del probs, p0, y
        torch.cuda.empty_cache()
        batch = batch_report(pipeline, torch, stream, args.wave_gb)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "value_definition": "2 E_t E^2 V,K entries per problem / assembly time (CUDA events "
                                "around every problem's stb_assemble call in the timed steps; "
                                "the best step, slowest rank)",
            "assembly_ms": {"best_step": asm_ms_best, "mean_step": asm_ms_mean,
                            "per_step": asm_ms_steps},
            "step_entries_per_s": step_rate,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if mixed else "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "E": E, "n_steps": n, "alphas": alphas,
                       "quad_regular": 3, "quad_singular": 4,
                       "nrhs": int(src.shape[0]),
                       "precision": "mixed (FP32 points, stated block error <= 2e-6; solve refined "
                                    "to 1e-10 with split-operand tensor-core residuals)"
                       if mixed else "fp64",
                       "storage": "f32" if mixed else "f64",
                       "l2": "no flush: every step writes %.1f GB of V/K blocks (>> 129 MB L2)"
                             % (2 * (4 if mixed else 8) * n * E * E * len(alphas) / 1e9),
                       "parallelism": "replicas" if world > 1 else "single"},
            "mixed_vs_fp64": cmp, "mixed_vs_fp64_sphere5120_e128": cmp3, "batch": batch, "matrix_free_rhs": mfree, "p1_data": p1,
            "neumann": neu,
            "potentials": pots, "nonuniform": nonuni,
            "matvec_tflops": mv_tflops, "matvec_ms": mv_ms, "matvec": matvec,
            "rel_l2_error_w": rel_err, "solve": solve_info,
            "timed_solves": [{"refinements": r, "rel_residual": res} for r, res, _ in solve_status],
            "concurrent_problems": concurrent, "gpu_launches": launches,
            "kernels_ms_first_problem_assembly": {k: v[1] for k, v in trace.items()},
            "roofline": roof,
            "measured_pipe_peaks": pipe_peaks, "e2e": e2e}
    if rank == 0:
        line["clocks"] = clk.summary()
        if world == 1 and not args.no_cpu_baseline:
            threads = host_threads()
            rate, rows, secs = cpu_oracle_rate(wl, alphas[0], args.cpu_seconds, threads)
            line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                    "sample": "%d whole rows (all %d blocks of V and K) of %s, "
                                              "alpha=%g, %.1f s on %d host threads"
                                              % (rows, n, args.workload, alphas[0], secs, threads)}
            rate1, rows1, secs1 = cpu_oracle_rate(wl, alphas[0], args.cpu_seconds / 4, 1)
            line["cpu_baseline_one_thread"] = {"value": rate1, "unit": UNIT, "cores": 1,
                                               "kind": "oracle",
                                               "sample": "%d whole rows, %.1f s" % (rows1, secs1)}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def batch_report(pipeline, torch, stream, wave_gb, runs=2):
    """The 64-problem batch (ellipsoids from seed 0) through the graph-captured
    batch pipeline, outside the headline's timed region: one warm-up run
    (builds and tunes the graphs), then `runs` timed runs of every wave's
    CUDA graph (batched assembly, projection, right-hand side, refined solve,
    error)."""
    probs = workloads.batch_workload(seed=0)
    bp = pipeline.BatchPipeline(probs, wave_bytes=wave_gb * 1e9)
    entries = sum(2.0 * len(p["tris"]) ** 2 * p["n_steps"] for p in probs)
    bp.run(stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(runs):
        bp.run(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / runs
    reports = bp.reports()
    errs = bp.relative_errors()
    out = {"workload": "batch64", "problems": len(probs), "waves": len(bp.waves),
           "wave_gb": wave_gb, "entries": entries, "ms_per_batch": ms,
           "entries_per_s": entries / (ms / 1e3),
           "timing": "CUDA events around %d replays of every wave's graph, after a warm-up run"
                     % runs,
           "refinements_max": max(r for r, _, _ in reports),
           "rel_residual_max": max(res for _, res, _ in reports),
           "solve_status": sorted(set(st for _, _, st in reports)),
           "rel_l2_error_w_range": [min(errs), max(errs)]}
    del bp
    torch.cuda.empty_cache()
    return out


def run_batch(args):
    """The 64-problem batch (ellipsoids from seed 0) through the graph-captured
    batch pipeline: every run replays one CUDA graph per memory wave."""
    import torch
    import torch.distributed as dist

    from paper_2102_09811_gb300 import capi, pipeline

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    probs = workloads.batch_workload(seed=0)
    bp = pipeline.BatchPipeline(probs, wave_bytes=args.wave_gb * 1e9)
    entries = sum(2.0 * len(p["tris"]) ** 2 * p["n_steps"] for p in probs)
    stream = torch.cuda.current_stream()
    for _ in range(max(1, args.warmup)):  # the first run builds and tunes the graphs
        bp.run(stream)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        barrier()
        start.record(stream)
        for _ in range(args.steps):
            bp.run(stream)
        end.record(stream)
        barrier()
    ms = max_over_ranks(start.elapsed_time(end), world, "cuda")
    value = whole_job_rate(entries, args.steps, ms, world)
    reports = bp.reports()
    errs = bp.relative_errors()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "value_definition": "2 E_t E^2 V,K entries summed over the 64 problems / time of "
                                "one whole batch (every wave's graph: assembly, projection, "
                                "right-hand side, refined solve, error)",
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch64", "problems": len(probs), "waves": len(bp.waves),
                       "wave_gb": args.wave_gb, "precision": "mixed, FP32 storage",
                       "graph": "one CUDA graph per wave (batched assembly, projection, RHS, "
                                "solve, error)",
                       "l2": "no flush: every step writes %.0f GB of V/K blocks" % (4 * entries / 1e9),
                       "parallelism": "replicas" if world > 1 else "single"},
            "gpu_launches": args.steps * sum(bp.graph_launches),
            "refinements_max": max(r for r, _, _ in reports),
            "rel_residual_max": max(res for _, res, _ in reports),
            "solve_status": sorted(set(st for _, _, st in reports)),
            "rel_l2_error_w_range": [min(errs), max(errs)], "e2e": None}
    if rank == 0:
        line["clocks"] = clk.summary()
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batch(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
