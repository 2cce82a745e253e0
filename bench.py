"""Benchmark: condensed-operator throughput and CG solve time to 1e-10, mixed vs FP64.

Workload (one step): one full solve of the 16^3 stretched-grid Helmholtz
problem (p = 8, lambda = 10, f ~ N(0, 1) per volume node) through hdg_solve
with device-resident inputs: transformed right-hand side, FP32 transformed CG
inside FP64 iterative refinement to ||F - K ut|| <= 1e-10 ||F|| (nodal
basis), traces back-transformed, u recovered.  L2 is flushed (a 256 MB
write) before every timed step.

value = trace DOFs solved per second (GDOF/s): the trace unknowns of the
problem divided by the time of one complete solve to 1e-10, summed over
ranks.  It does not grow with the number of operator applications a solve
needs; the operator's own rate (trace DOFs / operator launch time, live in
the solve and isolated) and trace DOFs x applications / solve time are
reported as secondary keys.  Each rank solves its own replica (different
seed): the mesh is not partitioned across GPUs ("scaling": "weak").

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import hdg_inputs  # noqa: E402

METRIC = "condensed-operator GDOF/s + CG solve time to 1e-10, mixed vs FP64 on 1 GB300"
WORKLOAD = "stretched_p8"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# FP64 FMA pipe derived from unit counts: 2 DFMA/clk/SM x 152 SMs x 2 flops x
# 2070 MHz; the bench measures the rate itself (hdg_measure_fma_peak, an FMA
# loop on every SM) and uses the measured value, this one only if that fails
FP64_PEAK_TFLOPS_DERIVED = 152 * 2 * 2 * 2.070e9 / 1e12
# DRAM bytes (read + write) per launch of the dominant kernel from one ncu
# capture of the same kernel and workload (cold caches); None when the
# kernel changed after the capture
TRAFFIC_BYTES = {"op_fp32": 6820608}   # tpt_fast_kernel<9, 1, float, 0> in the CG loop: read 6.82 MB, write 0


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return FALLBACK_PEAKS, "fallback"


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU reference (the oracle), bounded sample of the same workload
# ---------------------------------------------------------------------------
def oracle_sample(m):
    """Oracle solve on the m x m x m corner of the stretched 16^3 grid (same
    p, lambda, tau_hat, load distribution).  Returns (trace DOFs, operator
    applications, seconds)."""
    from oracle.solver import Problem
    cfg = hdg_inputs.WORKLOADS[WORKLOAD]
    grid = hdg_inputs.grid_lines(cfg["ne"], cfg["stretched"])
    sub = [g[:m + 1] for g in grid]
    t0 = time.perf_counter()
    pr = Problem((m, m, m), sub, (0,) * 6, cfg["p"], hdg_inputs.TAU_HAT, cfg["lam"])
    f = hdg_inputs.gaussian(pr.mesh.n_elem * (cfg["p"] + 1) ** 3, 11890)
    _, _, _, info = pr.solve(f=f, tol=1e-10)
    dt = time.perf_counter() - t0
    return pr.mesh.n_trace, info["iters"] + 1, dt


def cpu_baseline(m=3):
    T, applies, dt = oracle_sample(m)
    return {"value": T * applies / dt / 1e9, "unit": "GDOF/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "oracle solve (dense LU/Cholesky condensation per element, plain CG to 1e-10) on the "
                      "%dx%dx%d corner of the stretched 16^3 grid, p=8, lambda=10: %d trace DOFs, %d operator "
                      "applications, %.1f s; numpy/scipy BLAS threads up to cores" % (m, m, m, T, applies, dt)}


def run_reference(args, rank):
    if rank != 0:
        return
    m = 2
    for _ in range(args.warmup):
        oracle_sample(m)
    tot, work = 0.0, 0.0
    for _ in range(args.steps):
        T, applies, dt = oracle_sample(m)
        tot += dt
        work += T * applies
    value = work / tot / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "%s: oracle solve on the 2x2x2 corner of the 16^3 stretched grid, p=8, "
                                   "lambda=10, f~N(0,1), CG to 1e-10" % WORKLOAD},
            "cpu_baseline": {"value": value, "unit": "GDOF/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "2x2x2 corner of the stretched 16^3 grid per step"},
            "e2e": {"value": value, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def job_step_ms(ms_step, world, device):
    """Replicas: the job's step time is the slowest rank's (max over ranks)."""
    if world <= 1:
        return ms_step
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_step], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def solve_value(world, trace_dofs, ms_step):
    """Whole-job GDOF/s solved: every rank solves its own replica of
    `trace_dofs` unknowns to the tolerance within the job's step time."""
    return world * trace_dofs / (ms_step * 1e-3) / 1e9


def fp64_peak_tflops():
    """(FP64 FMA rate in TFLOP/s, where it comes from): measured on this GPU by
    the library's FMA loop, else derived from the unit counts."""
    try:
        from paper_2007_11891_gb300 import measure_fma_peak
        return measure_fma_peak("fp64"), "measured: FP64 FMA loop on every SM (hdg_measure_fma_peak)"
    except Exception:  # measurement unavailable: the unit-count figure
        return FP64_PEAK_TFLOPS_DERIVED, "derived: 2 DFMA/clk/SM x 152 SMs at 2070 MHz"


def job_value(world, trace_dofs, applies, ms_step):
    """Whole-job GDOF/s: every rank applies the operator `applies` times to
    its own replica's trace DOFs within the job's step time."""
    return world * trace_dofs * applies / (ms_step * 1e-3) / 1e9


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_2007_11891_gb300 import HDG

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    cfg = hdg_inputs.WORKLOADS[WORKLOAD]
    ne, p, lam = cfg["ne"], cfg["p"], cfg["lam"]
    grid = hdg_inputs.grid_lines(ne, cfg["stretched"])
    h = HDG(ne, grid, (0,) * 6, p, hdg_inputs.TAU_HAT)
    T, V = h.trace_size, h.volume_size
    f = torch.tensor(hdg_inputs.gaussian(V, 11890 + rank), device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(fn, steps):
        """Per-step CUDA-event time (ms) with an L2 flush before each step."""
        evs = []
        infos = None
        for _ in range(steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos = fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs), infos

    solve_mixed = lambda: h.solve(f, lam, tol=1e-10, inner="fp32")[2]
    solve_fp64 = lambda: h.solve(f, lam, tol=1e-10, inner="fp64")[2]

    for _ in range(args.warmup):
        solve_mixed()
    torch.cuda.synchronize()
    clk = ClockSampler(local_rank)
    clk.start()
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    ms, infos = timed(solve_mixed, args.steps)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - wall0
    clocks = clk.stop()
    applies = infos[0]["applies"]
    ms_step = job_step_ms(ms / args.steps, world, dev)

    # FP64 solve with the same machinery (FP64 inner CG)
    solve_fp64()
    n64 = max(2, args.steps // 5)
    ms64, infos64 = timed(solve_fp64, n64)
    ms64 /= n64

    # end to end through the public API with host buffers
    f_host = torch.empty(V, dtype=torch.float64, pin_memory=True)
    f_host.copy_(f.cpu())
    u_host = torch.empty(V, dtype=torch.float64, pin_memory=True)
    t_host = torch.empty(T, dtype=torch.float64, pin_memory=True)

    def e2e_step():
        fd = f_host.to(dev, non_blocking=True)
        tr, u, inf = h.solve(fd, lam, tol=1e-10, inner="fp32")
        u_host.copy_(u, non_blocking=True)
        t_host.copy_(tr, non_blocking=True)
        return inf

    e2e_step()
    ms_e2e, _ = timed(e2e_step, args.steps)
    ms_e2e = job_step_ms(ms_e2e / args.steps, world, dev)

    # isolated operator applications (transformed basis), L2 flushed per launch
    x64 = torch.tensor(hdg_inputs.uniform_pm1(T, 11893), device=dev)
    x32 = x64.float()
    app = {}
    for name, x in (("fp64", x64), ("fp32", x32)):
        y = torch.empty_like(x)
        for _ in range(3):
            h.apply(x, lam, basis="transformed", out=y)
        ms_a, _ = timed(lambda: h.apply(x, lam, basis="transformed", out=y), 20)
        app[name] = {"us": 1e3 * ms_a / 20, "gdofs": T / (ms_a / 20 * 1e-3) / 1e9}

    # live kernel timing inside one profiled mixed solve (events on the launch stream)
    h.profile(True)
    flush.fill_(1.0)
    _, _, pinfo = h.solve(f, lam, tol=1e-10, inner="fp32")
    classes = {}
    for k in h.KERNEL_CLASSES:
        tot_ms, cnt = h.profile_read(k)
        if cnt:
            classes[k] = {"ms": tot_ms, "launches": cnt}
    _, launches_per_solve = h.profile_read("all")
    h.profile(False)
    dominant = max(classes, key=lambda k: classes[k]["ms"])
    pk, src = peaks()
    fp64_peak, fp64_src = fp64_peak_tflops()
    n = p + 1
    ne_tot = ne[0] * ne[1] * ne[2]
    faces = T // (n * n)

    def alu(kind, name, flops, avg_s, note, pipe_ops=None):
        ach = flops / avg_s / 1e12
        out = {"kernel": name, "bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
               "frac": ach / fp64_peak, "traffic": None, "peak_source": fp64_src, "avg_launch_us": avg_s * 1e6,
               "algorithmic_flops_per_launch": flops, "flops_counted": note}
        if pipe_ops is not None:
            # FP64 pipe operations (an FMA, a multiply and an add each take one
            # issue slot of the pipe) against its rate, half the FMA flop rate
            out["fp64_pipe_ops_per_launch"] = pipe_ops
            out["frac_fp64_pipe_ops"] = pipe_ops / avg_s / (fp64_peak * 1e12 / 2.0)
        return out

    fp32_iters = pinfo[0]["iterations"] + pinfo[0]["outer"]   # operator applications of the inner CGs

    def roof(kind):
        c = classes[kind]
        avg_s = c["ms"] / c["launches"] * 1e-3
        if kind == "op_fp32":
            # the inner CG's operator kernel.  Fused step (no separate update
            # launches): per CG iteration it applies the previous update and
            # the operator, counted as the minimum bytes of a CG iteration.
            # Two kernels per iteration: the operator alone, 2 T values per
            # launch (read u, accumulate w), D_Z^-1 computed in the kernel.
            vec = classes.get("vector", {"ms": 0.0, "launches": 0})
            fused = vec["launches"] < fp32_iters // 2
            it_s = c["ms"] * 1e-3 / max(fp32_iters, c["launches"])
            pair_s = (c["ms"] + (0.0 if fused else vec["ms"])) * 1e-3 / max(fp32_iters, c["launches"])
            min_iter_b = 9.0 * T * 4
            op_b = 2.0 * T * 4
            byts = min_iter_b if fused else op_b
            ach = byts / it_s / 1e9
            name = ("FP32 fused CG step (operator + update in one launch per iteration)" if fused else
                    "tpt_fast_kernel<float> (FP32 operator of the inner CG, element runs)")
            return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / pk["hbm_gbs"], "traffic": None if fused else TRAFFIC_BYTES["op_fp32"],
                    "peak_source": "of " + src,
                    "launches_per_solve": c["launches"], "cg_iterations_per_solve": fp32_iters,
                    "avg_launch_us": it_s * 1e6, "algorithmic_bytes_per_launch": byts,
                    "bytes_counted": ("9 T x 4 B per CG iteration, the minimum of a CG iteration (operator: read "
                                      "x, write y; vectors: read r, p, Ap, x, write r, p, x)" if fused else
                                      "2 T x 4 B per launch: read the input u, write the output w (each face "
                                      "value read by its two elements counts once); D_Z^-1 computed in the "
                                      "kernel (0 table bytes)"),
                    "cg_iteration": {"us": pair_s * 1e6, "min_bytes": min_iter_b,
                                     "frac": min_iter_b / pair_s / 1e9 / pk["hbm_gbs"],
                                     "note": "operator + update per CG iteration against the minimum bytes of "
                                             "a CG iteration (9 T x 4 B)"}}
        if kind == "op_fp64":
            return alu(kind, "tpt_tile_kernel<double> (operator, FP64, refinement residual)",
                       (12.0 * n ** 3 + 24.0 * n ** 2) * ne_tot, avg_s,
                       "executed: 12 n^3 + 24 n^2 per element (parity-split expansion and contraction); "
                       "pipe operations 7 n^3 + 42 n^2 per element",
                       pipe_ops=(7.0 * n ** 3 + 42.0 * n ** 2) * ne_tot)
        if kind == "face":
            return alu(kind, "face_rows_kernel (FP64 face transforms)", 2.0 * n ** 3 * faces, avg_s,
                       "executed: 2 n^3 per face (parity-split line transforms, rows and columns)")
        if kind == "volume":
            return alu(kind, "volume_transform_kernel (FP64)", 3.0 * n ** 4 * ne_tot, avg_s,
                       "executed: 3 n^4 per element (parity-split line transforms along three directions)")
        if kind == "rhs_recover":
            return alu(kind, "tpt_kernel<double> RHS / RECOVER modes", (13.0 * n ** 3 + 24.0 * n ** 2) * ne_tot,
                       avg_s, "executed: 13 n^3 + 24 n^2 per element")
        byts = 12.0 * T * 4
        ach = byts / avg_s / 1e9
        return {"kernel": "CG vector kernels (cg_step_kernel<float> and the solve's other vector launches)",
                "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": ach / pk["hbm_gbs"],
                "traffic": None, "peak_source": "of " + src, "avg_launch_us": avg_s * 1e6,
                "bytes_counted": "12 streams of T FP32 values per launch (cg_step_kernel reads w, p, s, x, r, W "
                                 "and writes p, s, x, r, u, w); the average includes the few other vector launches"}

    roofline = roof(dominant)
    roofline["share_of_solve"] = classes[dominant]["ms"] / sum(c["ms"] for c in classes.values())
    others = {k: roof(k) for k in classes if k != dominant}
    op_live = classes.get("op_fp32")

    line = {
        "metric": METRIC, "value": solve_value(world, T, ms_step), "unit": "GDOF/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "%s: 16x16x16 stretched grid (widths U[0.5,2], seeded), p=8, lambda=10, "
                               "tau_hat=25, Dirichlet, f~N(0,1); one full mixed-precision solve per step "
                               "(FP32 transformed CG inside FP64 refinement) to 1e-10" % WORKLOAD,
                   "value": "trace DOFs / time of one solve to 1e-10 (summed over ranks)",
                   "trace_dofs": T, "volume_dofs": V, "l2": "flushed before each step (256 MB write)",
                   "parallelism": "replicas (one independent solve per GPU)"},
        "clocks": clocks,
        "e2e": {"value": solve_value(world, T, ms_e2e), "unit": "GDOF/s",
                "h2d_bytes_per_step": V * 8, "d2h_bytes_per_step": (V + T) * 8, "ms_per_step": ms_e2e},
        "gpu_launches": launches_per_solve * args.steps,
        "roofline": roofline,
        "roofline_other_kernels": others,
        "solve": {"mixed_ms": ms_step, "fp64_ms": ms64, "speedup_mixed_vs_fp64": ms64 / ms_step,
                  "mixed": infos[0], "fp64": infos64[0], "wall_s_timed": wall},
        "operator_gdofs": {
            "live_fp32_in_solve_per_cg_iteration": (T / (op_live["ms"] * 1e-3 / max(fp32_iters, op_live["launches"]))
                                                    / 1e9) if op_live else None,
            "isolated_fp32": app["fp32"]["gdofs"], "isolated_fp64": app["fp64"]["gdofs"],
            "applications_x_trace_dofs_per_solve_time": job_value(world, T, applies, ms_step)},
        "apply_isolated_transformed": app,
        "kernel_time_by_class_ms": classes,
    }
    if rank == 0:
        if world == 1:
            try:
                line["cpu_baseline"] = cpu_baseline()
            except Exception as exc:  # the oracle is optional on the GPU machine
                line["cpu_baseline"] = {"value": None, "unit": "GDOF/s", "kind": "oracle", "error": str(exc)}
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# extra measurements (not the contract line): operator sweep and batched solve
# ---------------------------------------------------------------------------
def run_sweep(args):
    """One JSON line per measurement: the 32^3 operator sweep (p in
    {2, 4, 8, 12, 16}, FP64 and FP32, transformed basis, L2 flushed per
    launch) against its roofline, the paper's manufactured solver test
    (8^3 on (0, 2 pi)^3, lambda = 0, p = 2..32: iterations, error, time per
    unknown), the BF16-stored apply (32^3, p = 8), the adjoint solve (32^3,
    p = 6), and the 64-rhs batched solve (24^3, p = 7, lambda from
    {0.1, 1, 100}) mixed vs FP64; also the nodal-basis FP64 apply at 32^3
    (face-wise transforms against one kernel per apply) and the 1D/2D
    operators.  ``--parts``
    selects sections."""
    import torch
    from paper_2007_11891_gb300 import HDG
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    pk, src = peaks()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def per_launch_ms(fn, reps):
        for _ in range(3):   # warm-up: first-use costs (module loading, attributes) stay out
            fn()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(reps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / reps

    parts = set(args.parts.split(","))
    fp64_peak, fp64_src = fp64_peak_tflops()
    fp32_peak = None
    try:
        from paper_2007_11891_gb300 import measure_fma_peak
        fp32_peak = measure_fma_peak("fp32")
    except Exception:  # measurement unavailable
        pass
    print(json.dumps({"sweep": "peaks", "fp64_tflops": fp64_peak, "fp64_source": fp64_src,
                      "fp32_fma_loop_tflops": fp32_peak, "hbm_gbs": pk["hbm_gbs"], "hbm_source": src}), flush=True)
    if "operator" in parts:
        cfg = hdg_inputs.WORKLOADS["uniform32"]
        ne = cfg["ne"]
        grid = hdg_inputs.grid_lines(ne)
        for p in (2, 4, 8, 12, 16):
            h = HDG(ne, grid, (0,) * 6, p, hdg_inputs.TAU_HAT)
            T = h.trace_size
            n = p + 1
            x64 = torch.tensor(hdg_inputs.uniform_pm1(T, 11893), device=dev)
            for prec, x in (("fp64", x64), ("fp32", x64.float())):
                y = torch.empty_like(x)
                h.apply(x, cfg["lam"], basis="transformed", out=y)
                ms = per_launch_ms(lambda: h.apply(x, cfg["lam"], basis="transformed", out=y), 10)
                line = {"sweep": "operator", "workload": "uniform32", "p": p, "precision": prec,
                        "trace_dofs": T, "us_per_apply": ms * 1e3, "gdofs": T / (ms * 1e-3) / 1e9}
                if prec == "fp32":
                    ach = 2.0 * T * 4 / (ms * 1e-3) / 1e9
                    line["roofline"] = {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                                        "frac": ach / pk["hbm_gbs"], "peak_source": "of " + src}
                else:
                    flops = (12.0 * n ** 3 + 24.0 * n ** 2) * ne[0] * ne[1] * ne[2]
                    ach = flops / (ms * 1e-3) / 1e12
                    line["roofline"] = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                                        "frac": ach / fp64_peak, "peak_source": fp64_src}
                print(json.dumps(line), flush=True)
            h.close()
            del x64
    if "nodal" in parts:
        # nodal-basis FP64 apply, 32^3 uniform: face-wise transforms around the
        # transformed kernel (three launches) against one kernel per apply
        # (Alg. hdg_op_3d, each element transforms its own faces)
        cfg = hdg_inputs.WORKLOADS["uniform32"]
        ne = cfg["ne"]
        grid = hdg_inputs.grid_lines(ne)
        for p in (2, 4, 8, 12, 16):
            h = HDG(ne, grid, (0,) * 6, p, hdg_inputs.TAU_HAT)
            T = h.trace_size
            n = p + 1
            nel = ne[0] * ne[1] * ne[2]
            x = torch.tensor(hdg_inputs.uniform_pm1(T, 11893), device=dev)
            y = torch.empty_like(x)
            # executed flops per element: face-wise = parity-split face transforms
            # in and out (2 n^3 each, three faces per element) around the
            # transformed core (12 n^3 + 24 n^2); one kernel = dense transforms
            # of all six faces in and out (48 n^3) around the same core
            for variant, fl in (("facewise", 24.0 * n ** 3 + 24.0 * n ** 2), ("fused", 60.0 * n ** 3 + 24.0 * n ** 2)):
                h.set_nodal_variant(variant)
                h.apply(x, cfg["lam"], basis="nodal", out=y)
                ms = per_launch_ms(lambda: h.apply(x, cfg["lam"], basis="nodal", out=y), 5)
                ach = fl * nel / (ms * 1e-3) / 1e12
                print(json.dumps({"sweep": "nodal_apply", "workload": "uniform32", "p": p, "variant": variant,
                                  "trace_dofs": T, "us_per_apply": ms * 1e3, "gdofs": T / (ms * 1e-3) / 1e9,
                                  "flops_per_element": fl,
                                  "roofline": {"bound": "alu", "achieved": ach, "peak": fp64_peak,
                                               "unit": "TFLOP/s", "frac": ach / fp64_peak,
                                               "peak_source": fp64_src}}), flush=True)
            h.close()
            del x, y
    if "lowdim" in parts:
        # 1D (Alg. hdg_op_1d) and 2D operators, FP64, uniform grids, lambda = 1,
        # Dirichlet sides: 10^6 elements at p = 8 (1D), 512 x 512 at p = 8 (2D)
        from paper_2007_11891_gb300 import HDGLowDim
        for ne in ((1000000,), (512, 512)):
            p = 8
            grid = [np.linspace(0.0, 1.0, v + 1) for v in ne]
            h = HDGLowDim(ne, grid, (0,) * (2 * len(ne)), p, hdg_inputs.TAU_HAT)
            T = h.trace_size
            nel = int(np.prod(ne))
            x = torch.tensor(hdg_inputs.uniform_pm1(T, 11893), device=dev)
            y = torch.empty_like(x)
            for basis in ("nodal", "transformed") if len(ne) == 2 else ("nodal",):
                h.apply(x, 1.0, basis=basis, out=y)
                ms = per_launch_ms(lambda: h.apply(x, 1.0, basis=basis, out=y), 10)
                byt = 2.0 * T * 8 + 32.0 * nel   # traces in and out, metric factors
                ach = byt / (ms * 1e-3) / 1e9
                print(json.dumps({"sweep": "lowdim_apply", "dim": len(ne), "ne": list(ne), "p": p, "basis": basis,
                                  "trace_dofs": T, "us_per_apply": ms * 1e3, "gdofs": T / (ms * 1e-3) / 1e9,
                                  "roofline": {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                                               "frac": ach / pk["hbm_gbs"], "peak_source": "of " + src}}), flush=True)
            h.close()
            del x, y
    if "paper" in parts:
        # the paper's solver test (Sec. 5.3): 8^3 elements on (0, 2 pi)^3, lambda = 0,
        # inhomogeneous Dirichlet data from u_ex (k = 5), residual reduced by 1e-10
        cfg = hdg_inputs.WORKLOADS["paper_case"]
        ne = cfg["ne"]
        grid = hdg_inputs.grid_lines(ne, length=cfg["length"])
        for p in range(2, 33):
            h = HDG(ne, grid, (0,) * 6, p, hdg_inputs.TAU_HAT)
            X = h.volume_coords()
            f = torch.tensor(hdg_inputs.paper_case_load(X, cfg["lam"]), device=dev)
            bd = torch.tensor(hdg_inputs.paper_case_u(h.boundary_coords()[0]), device=dev)
            uex = hdg_inputs.paper_case_u(X)
            for inner in ("fp32", "fp64"):
                run = lambda: h.solve(f, cfg["lam"], bdry=bd, tol=1e-10, inner=inner)
                run()
                ms = per_launch_ms(run, 3)
                _, u, info = run()
                T = h.trace_size
                print(json.dumps({"sweep": "paper_case", "workload": "paper_case", "p": p, "inner": inner,
                                  "trace_dofs": T, "ms": ms, "iterations": info[0]["iterations"],
                                  "outer": info[0]["outer"], "rel_residual": info[0]["rel_residual"],
                                  "status": info[0]["status"],
                                  "max_error": float(np.abs(u.cpu().numpy() - uex).max()),
                                  "ns_per_unknown": ms * 1e6 / T,
                                  "ns_per_unknown_iteration": ms * 1e6 / T / max(info[0]["iterations"], 1)}),
                      flush=True)
            h.close()
    if "bf16" in parts:
        # BF16-stored operator (transformed basis), 32^3, p = 8: FP32 arithmetic, half the bytes
        cfg = hdg_inputs.WORKLOADS["uniform32"]
        ne = cfg["ne"]
        h = HDG(ne, hdg_inputs.grid_lines(ne), (0,) * 6, 8, hdg_inputs.TAU_HAT)
        xb = torch.tensor(hdg_inputs.uniform_pm1(h.trace_size, 11893), device=dev).to(torch.bfloat16)
        yb = torch.empty_like(xb)
        h.apply(xb, cfg["lam"], basis="transformed", out=yb)
        ms = per_launch_ms(lambda: h.apply(xb, cfg["lam"], basis="transformed", out=yb), 10)
        ach = 2.0 * h.trace_size * 2 / (ms * 1e-3) / 1e9
        print(json.dumps({"sweep": "operator", "workload": "uniform32", "p": 8, "precision": "bf16-stored",
                          "trace_dofs": h.trace_size, "us_per_apply": ms * 1e3,
                          "gdofs": h.trace_size / (ms * 1e-3) / 1e9,
                          "roofline": {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                                       "frac": ach / pk["hbm_gbs"], "peak_source": "of " + src}}), flush=True)
        h.close()
        del xb, yb
    if "adjoint" in parts:
        # adjoint (32^3, p = 6, lambda = 5): forward solve, L = ||u - u_t||^2, adjoint solve
        cfg = hdg_inputs.WORKLOADS["adjoint32_p6"]
        ne, p = cfg["ne"], cfg["p"]
        h = HDG(ne, hdg_inputs.grid_lines(ne), (0,) * 6, p, hdg_inputs.TAU_HAT)
        f = torch.tensor(hdg_inputs.gaussian(h.volume_size, 11897), device=dev)
        ut = torch.tensor(hdg_inputs.smooth_target(h.volume_coords(), hdg_inputs.smooth_target_coeffs()), device=dev)
        for inner in ("fp32", "fp64"):
            fwd = lambda: h.solve(f, cfg["lam"], tol=1e-10, inner=inner)
            _, u, info_f = fwd()
            ms_f = per_launch_ms(fwd, 2)
            gu = 2.0 * (u - ut)
            adj = lambda: h.solve_adjoint(u, gu, cfg["lam"], tol=1e-10, inner=inner)
            _, gl, info_a = adj()
            ms_a = per_launch_ms(adj, 2)
            print(json.dumps({"sweep": "adjoint", "workload": "adjoint32_p6", "inner": inner, "trace_dofs": h.trace_size,
                              "forward_ms": ms_f, "adjoint_ms": ms_a, "forward_iterations": info_f[0]["iterations"],
                              "adjoint_iterations": info_a[0]["iterations"],
                              "loss": float(((u - ut) ** 2).sum()), "dL_dlambda": float(gl[0]),
                              "status": [info_f[0]["status"], info_a[0]["status"]]}), flush=True)
        h.close()
    if "batched" in parts:
        # batched solve
        cfg = hdg_inputs.WORKLOADS["batched24_p7"]
        ne, p, nrhs = cfg["ne"], cfg["p"], cfg["nrhs"]
        h = HDG(ne, hdg_inputs.grid_lines(ne), (0,) * 6, p, hdg_inputs.TAU_HAT)
        lams = hdg_inputs.batch_lambdas(nrhs)
        F = torch.tensor(np.stack([hdg_inputs.gaussian(h.volume_size, 11894 + r) for r in range(nrhs)]), device=dev)
        for inner in ("fp32", "fp64"):
            h.solve(F, lams, tol=1e-10, inner=inner)
            ms = per_launch_ms(lambda: h.solve(F, lams, tol=1e-10, inner=inner), 2)
            _, _, info = h.solve(F, lams, tol=1e-10, inner=inner)
            print(json.dumps({"sweep": "batched_solve", "workload": "batched24_p7", "nrhs": nrhs, "inner": inner,
                              "ms": ms, "trace_dofs_per_rhs": h.trace_size,
                              "max_iterations": max(i["iterations"] for i in info),
                              "max_rel_residual": max(i["rel_residual"] for i in info),
                              "all_ok": all(i["status"] == "OK" for i in info)}), flush=True)


def run_probe(args):
    """Short, untimed workload for ncu captures: set-up, one warm-up, then
    `--steps` repetitions of the probed step on the chosen workload:
      solve            mixed solve (CG iteration per --cg-variant)
      solve_two_kernel mixed solve with the operator + update kernel pair
      solve_fp64       solve with the FP64 inner CG
      apply32/64/bf16  one transformed-basis operator application
      nodal_fused      one nodal FP64 apply by the one-kernel HDG-TP operator
      lowdim2          one 2D operator application (512 x 512 elements, p = 8)
    With --eager the solve launches its kernels one by one (the same kernels
    as inside the CUDA graph)."""
    import torch
    from paper_2007_11891_gb300 import HDG, HDGLowDim
    torch.cuda.set_device(0)
    cfg = hdg_inputs.WORKLOADS[args.workload]
    ne, p, lam = cfg["ne"], cfg["p"], cfg["lam"] or 1.0
    if args.degree:
        p = args.degree
    if args.probe == "lowdim2":
        ne2 = (512, 512)
        h = HDGLowDim(ne2, [np.linspace(0.0, 1.0, v + 1) for v in ne2], (0,) * 4, 8, hdg_inputs.TAU_HAT)
        x = torch.tensor(hdg_inputs.uniform_pm1(h.trace_size, 11893), device="cuda")
        y = torch.empty_like(x)
        step = lambda: h.apply(x, 1.0, basis="transformed", out=y)
    else:
        h = HDG(ne, hdg_inputs.grid_lines(ne, cfg["stretched"]), (0,) * 6, p, hdg_inputs.TAU_HAT)
        h.set_operator_variant(args.op_variant)
        h.set_cg_variant(args.cg_variant)
        if args.eager:
            h.profile(True)   # per-launch events; keeps the solver off CUDA graphs
        if args.probe in ("solve", "solve_two_kernel", "solve_fp64"):
            if args.probe == "solve_two_kernel":
                h.set_cg_variant("two_kernel")
            f = torch.tensor(hdg_inputs.gaussian(h.volume_size, 11890), device="cuda")
            inner = "fp64" if args.probe == "solve_fp64" else "fp32"
            step = lambda: h.solve(f, lam, tol=1e-10, inner=inner, return_u=True)
        elif args.probe == "nodal_fused":
            h.set_nodal_variant("fused")
            x = torch.tensor(hdg_inputs.uniform_pm1(h.trace_size, 11893), device="cuda")
            y = torch.empty_like(x)
            step = lambda: h.apply(x, lam, basis="nodal", out=y)
        else:
            dt = {"apply32": torch.float32, "apply64": torch.float64, "apply_bf16": torch.bfloat16}[args.probe]
            x = torch.tensor(hdg_inputs.uniform_pm1(h.trace_size, 11893), device="cuda").to(dt)
            y = torch.empty_like(x)
            step = lambda: h.apply(x, lam, basis="transformed", out=y)
    step()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    print("probe done", args.probe, args.workload, h.trace_size)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sweep", action="store_true", help="extra measurements instead of the bench line")
    ap.add_argument("--parts", default="operator,nodal,lowdim,paper,bf16,adjoint,batched",
                    help="sweep sections to run (comma-separated)")
    ap.add_argument("--probe", choices=["solve", "solve_two_kernel", "solve_fp64", "apply32", "apply64",
                                        "apply_bf16", "nodal_fused", "lowdim2"], help="untimed workload for ncu")
    ap.add_argument("--op-variant", default="auto", choices=["auto", "runs", "tiles", "generic"],
                    help="probe: operator kernel (hdg_set_operator_variant)")
    ap.add_argument("--cg-variant", default="auto", choices=["auto", "persistent", "fused", "two_kernel"],
                    help="probe: inner CG iteration (hdg_set_cg_variant)")
    ap.add_argument("--degree", type=int, default=0, help="probe: polynomial degree instead of the workload's")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(hdg_inputs.WORKLOADS))
    ap.add_argument("--eager", action="store_true",
                    help="probe: launch the CG loop kernel by kernel (no CUDA graphs), so that profilers that "
                         "cannot enter conditional graph nodes see every launch")
    args = ap.parse_args()
    if args.probe:
        run_probe(args)
        return
    if args.sweep:
        run_sweep(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
