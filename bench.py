"""Benchmark of the space-time heat BEM hot path on GB300.

One step = one pass of the whole path for every heat capacity constant of
the workload: triangle geometry and pair classification, assembly of all
blocks V^d and K^d, Dirichlet data projection, right-hand side
(1/2 M_h + K_h) g, forward-substitution solve and the L2(Sigma_h) error.
Metric: V,K block entries produced per second (2 E_t E^2 per problem).

Default workload: cube surface with 16 x 16 squares per face (3072
triangles), 64 uniform steps on T = 1, alpha in {0.5, 1, 2}, exterior heat
source (1.5, 1.5, 1.5), t0 = 0.

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
FP64_FLOPS_PER_EVAL = None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", default="cube3072_e64")
    ap.add_argument("--alphas", default="0.5,1,2")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


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


def cpu_oracle_rate(wl, alpha, seconds):
    """The FP64 oracle (single thread) on whole rows of V and K: entries/s."""
    import oracle
    E, n = len(wl["tris"]), wl["n_steps"]
    rows_done, t_used, row = 0, 0.0, 0
    while t_used < seconds and rows_done < E:
        t0 = time.perf_counter()
        oracle.assemble_rows(wl["nodes"], wl["tris"], alpha, wl["T"], n, np.array([row]))
        t_used += time.perf_counter() - t0
        rows_done += 1
        row = (row + 977) % E
    return 2.0 * n * E * rows_done / t_used, rows_done, t_used


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    wl = workloads.workload(args.workload)
    alphas = [float(a) for a in args.alphas.split(",")]
    E, n = len(wl["tris"]), wl["n_steps"]
    per_step = max(1.0, args.cpu_seconds / 3.0)
    for i in range(args.warmup):
        cpu_oracle_rate(wl, alphas[i % len(alphas)], per_step / 4)
    rates, rows_total, secs_total = [], 0, 0.0
    for i in range(args.steps):
        r, rows, secs = cpu_oracle_rate(wl, alphas[i % len(alphas)], per_step)
        rates.append(r)
        rows_total += rows
        secs_total += secs
    value = 2.0 * n * E * rows_total / secs_total
    sample = "%d whole rows (all %d blocks of V and K) of %s, alpha cycling %s" % (
        rows_total, n, args.workload, alphas)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * 2 * n * E * E * len(alphas) / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "E": E, "n_steps": n, "alphas": alphas,
                       "quad_regular": 3, "quad_singular": 4},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2102_09811_gb300 import capi, pipeline

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    wl = workloads.workload(args.workload)
    alphas = [float(a) for a in args.alphas.split(",")]
    E, n = len(wl["tris"]), wl["n_steps"]
    nodes, tris, src = wl["nodes"], wl["tris"], wl["sources"]
    mesh = capi.Mesh(nodes, tris)
    probs = [pipeline.DirichletProblem(nodes, tris, a, wl["T"], n, src, mesh=mesh) for a in alphas]
    stream = torch.cuda.current_stream()

    def step():
        for p in probs:
            p.run(stream)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    capi.stb_trace_enable(True)
    capi.stb_trace_reset()
    launches0 = capi.stb_launch_count()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        barrier()
        start.record(stream)
        for _ in range(args.steps):
            step()
        end.record(stream)
        barrier()
    capi.stb_trace_enable(False)
    launches = capi.stb_launch_count() - launches0
    trace = capi.stb_trace_read()
    ms = start.elapsed_time(end)
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    entries = 2.0 * n * E * E * len(alphas)
    value = world * entries * args.steps / (ms / 1e3)
    rel_err = [p.relative_error() for p in probs]

    # block-Toeplitz matvec (FP64) on the assembled V of the first problem
    p0 = probs[0]
    ws = torch.empty(capi.stb_toeplitz_workspace_size(E, n, p0.nrhs), dtype=torch.uint8, device="cuda")
    y = torch.empty_like(p0.w)
    capi.stb_toeplitz_matvec(p0.V, capi.STB_STORE_F64, E, n, p0.nrhs, p0.w, 0.0, y, ws)
    torch.cuda.synchronize()
    a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    a_.record(stream)
    for _ in range(reps):
        capi.stb_toeplitz_matvec(p0.V, capi.STB_STORE_F64, E, n, p0.nrhs, p0.w, 0.0, y, ws)
    b_.record(stream)
    torch.cuda.synchronize()
    mv_ms = a_.elapsed_time(b_) / reps
    mv_tflops = float(E) * E * n * (n + 1) * p0.nrhs / (mv_ms / 1e3) / 1e12

    # end to end through the public API from host buffers (mesh, sources in;
    # solution and error norms out)
    e2e = None
    if not args.no_e2e:
        h2d = d2h = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(max(1, min(args.steps, 2))):
            for a in alphas:
                pr = pipeline.DirichletProblem(nodes, tris, a, wl["T"], n, src)
                pr.run(stream)
                w_host = pr.w.cpu()
                err_host = pr.err.cpu()
                h2d += nodes.nbytes + tris.nbytes + src.nbytes
                d2h += w_host.numel() * 8 + err_host.numel() * 8
                del pr
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        n_e2e = max(1, min(args.steps, 2))
        e2e = {"value": world * entries * n_e2e / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": h2d // n_e2e, "d2h_bytes_per_step": d2h // n_e2e}

    # roofline of the dominant kernel from the live trace
    name, (cnt, tot) = max(trace.items(), key=lambda kv: kv[1][1])
    n_reg_pairs = E * E - mesh.n_touching * 2 + E  # ordered separated pairs
    q2 = 3 * 3
    evals = float(n_reg_pairs) * q2 * q2 * n  # levels 1..E_t per launch
    roof = {"kernel": name, "bound": "alu", "unit": "TFLOP/s", "peak": FP64_PEAK_TFLOPS,
            "peak_source": "derived: 152 SM x 2 FP64 FMA/clk x 2.07 GHz (nominal FP64 1.25 TFLOP/s)",
            "launch_ms": tot / cnt, "share_of_step": tot / ms, "evaluations_per_launch": evals,
            "traffic": None}
    if name == "k_regular_f64" and FP64_FLOPS_PER_EVAL:
        achieved = FP64_FLOPS_PER_EVAL * evals / (tot / cnt / 1e3) / 1e12
        roof.update({"achieved": achieved, "frac": achieved / FP64_PEAK_TFLOPS})
    else:
        roof.update({"achieved": None, "frac": None,
                     "evals_per_s": evals / (tot / cnt / 1e3)})

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "E": E, "n_steps": n, "alphas": alphas,
                       "quad_regular": 3, "quad_singular": 4, "precision": "fp64",
                       "l2": "no flush: every step writes %.1f GB of V/K blocks (>> 129 MB L2)"
                             % (2 * 8 * n * E * E * len(alphas) / 1e9),
                       "parallelism": "replicas" if world > 1 else "single"},
            "matvec_tflops": mv_tflops, "matvec_ms": mv_ms,
            "rel_l2_error_w": rel_err, "gpu_launches": launches,
            "kernels_ms": {k: v[1] for k, v in trace.items()}, "roofline": roof, "e2e": e2e}
    if rank == 0:
        line["clocks"] = clk.summary()
        if world == 1 and not args.no_cpu_baseline:
            rate, rows, secs = cpu_oracle_rate(wl, alphas[0], args.cpu_seconds)
            line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": "%d whole rows (all %d blocks of V and K) of %s, "
                                              "alpha=%g, %.1f s" % (rows, n, args.workload,
                                                                     alphas[0], secs)}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
