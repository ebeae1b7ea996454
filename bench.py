"""Benchmark of the tensor-product--Thomas solve on GB300.

Workload (one step = one complete solve): Poisson on a 512x512x512
staggered grid, tanh-stretched in x, y, z with factors 1.5 / 2.0 / 2.5,
homogeneous Neumann walls, x and y by eigenbasis GEMM, z by Thomas, seeded
uniform[-1, 1] right-hand side with its volume-weighted mean removed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision fp64|mixed_bf16x3|...] [--size 512]

Prints one JSON line.  The solver is a one-GPU program: its transform GEMMs
may pair two CTAs that share an operand tile by TMA multicast within this
GPU's own memory, and the path has no exchange step to shard, so ``--gpus``
other than 1 (or a launch under torchrun with WORLD_SIZE > 1) is refused
with a message and exit status 2.  The timed region is bracketed by a device
synchronisation on both sides.  ``--impl reference`` times the CPU oracle
(the reference arm of this project) on the host cores on a bounded sample of
the same workload; under torchrun only rank 0 runs it and the others exit 0.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Poisson solves/s & Gpts/s at 512³ stretched, FP64 vs mixed+refine; p99 latency"
STRETCH = (1.5, 2.0, 2.5)
SEED = 4


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 20 ms from before
    the warm-up (so that the sampler is running when the timed region starts)
    to after the timed region; stop() keeps the samples taken inside the
    timed window (its start and end marked with mark()), widened by one
    sampling period, and counts the rest separately."""
    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_S = 0.02

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self._t = None
        self.window = [None, None]

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", str(int(self.PERIOD_S * 1000))],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def mark(self, i):
        import datetime
        self.window[i] = datetime.datetime.now()

    def stop(self):
        import datetime
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self._t.join(timeout=2)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = self.window
        pad = datetime.timedelta(seconds=self.PERIOD_S)
        inside, outside = [], 0
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
                row = (float(parts[2]), float(parts[3]), float(parts[4]) if parts[4] else float("nan"),
                       {nm for nm, v in zip(names, parts[6:10]) if v.lower() == "active"})
            except ValueError:
                continue
            if t0 is not None and t1 is not None and t0 - pad <= ts <= t1 + pad:
                inside.append(row)
            else:
                outside += 1
        if not inside:
            return None
        return {"sm_mhz": float(np.median([r[0] for r in inside])), "sm_max_mhz": float(max(r[1] for r in inside)),
                "power_w": float(np.median([r[2] for r in inside])),
                "reasons": sorted(set().union(*[r[3] for r in inside])), "samples": len(inside),
                "period_ms": self.PERIOD_S * 1e3, "samples_outside_window": outside}


# ------------------------------------------------------------------ inputs

def workload(size):
    n = (size, size, size)
    return n, STRETCH


def workload_name(size):
    if size == 512:
        return "poisson_512cube_tanh1.5-2.0-2.5_neumann_GG_thomas"
    return "poisson_%dcube_tanh1.5-2.0-2.5_neumann" % size


def rhs_host(n, grids):
    import seeded_inputs as S
    f = S.uniform_rhs(n, SEED)
    return S.remove_weighted_mean(f, [g[0] for g in grids])


# ------------------------------------------------------------- reference arm

def cpu_sample(n, nslab, reps=1):
    """Times the oracle on a bounded sample of the workload: one correction
    pass (forward x, forward y, Thomas, inverse y, inverse x) plus one residual
    on an Nx x Ny x nslab slab of the same stretched grid, repeated ``reps``
    times; returns seconds per full-size refined solve (two passes and two
    residuals over all Nz slabs), scaled by points."""
    import oracle as O
    import seeded_inputs as S
    nz_full = n[2]
    dirs = O.make_dirs((n[0], n[1], nslab), STRETCH, [(O.NEUMANN, O.NEUMANN)] * 3)
    f = S.remove_weighted_mean(S.uniform_rhs((n[0], n[1], nslab), SEED), [d.dxf for d in dirs])
    solver = O.TensorSolver(dirs, 0.0, 1.0)
    best = None
    for _ in range(reps):
        t0 = time.perf_counter()
        phi = solver.direct(f)
        O.residual(f, phi, dirs, 0.0, 1.0)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    per_point = best / (n[0] * n[1] * nslab)
    return 2.0 * per_point * n[0] * n[1] * nz_full


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def cpu_single_thread(size, nslab):
    """cpu_sample in a child process with one BLAS/OpenMP thread; seconds per
    full-size refined solve, or None if the child fails."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, os.path.abspath(__file__), "--size", str(size),
                              "--cpu-sample-only", str(nslab)], capture_output=True, text=True, env=env,
                             timeout=600)
        return float(out.stdout.strip().splitlines()[-1])
    except Exception:
        return None


def cpu_baseline_record(n, size, nslab, s_per_solve):
    """The cpu_baseline object: the oracle at the host's BLAS threads on an
    nslab-plane slab, plus the same sample on one thread (a 1/16 slab)."""
    rec = {"value": 1.0 / s_per_solve, "unit": "solves/s", "cores": _threads(), "kind": "oracle",
           "cpu": cpu_model(),
           "sample": "oracle (numpy float64) correction pass + residual on a %dx%dx%d slab of the "
                     "%d^3 stretched Neumann grid, scaled by points to one refined solve "
                     "(2 passes + 2 residuals)" % (n[0], n[1], nslab, n[2])}
    slab1 = max(1, nslab // 16)
    t1 = cpu_single_thread(size, slab1)
    if t1:
        rec["single_thread"] = {"value": 1.0 / t1, "unit": "solves/s", "cores": 1,
                                "sample": "the same on a %dx%dx%d slab, one BLAS thread" % (n[0], n[1], slab1)}
    return rec


def _threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    rank = _env_int("RANK", 0)
    if not runs_reference_leg(rank):
        return 0
    n, _ = workload(args.size)
    nslab = max(1, min(n[2], args.cpu_slabs))
    for _ in range(args.warmup):
        cpu_sample(n, nslab)
    times = [cpu_sample(n, nslab) for _ in range(args.steps)]
    s_per_solve = float(np.mean(times))
    val = 1.0 / s_per_solve
    sample = ("oracle (numpy float64) correction pass + residual on a %dx%dx%d slab of the "
              "%d^3 stretched Neumann grid, scaled by points to one refined solve "
              "(2 passes + 2 residuals)" % (n[0], n[1], nslab, n[2]))
    cpu = cpu_baseline_record(n, args.size, nslab, s_per_solve)
    out = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": s_per_solve * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.size), "size": list(n),
                   "sample": "z-slab of %d" % nslab},
        "gpts_per_s": val * n[0] * n[1] * n[2] / 1e9,
        "cpu_baseline": dict(cpu, sample=sample),
        "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)
    return 0


# --------------------------------------------------------------- our arm

PRECISIONS = {"fp64": 0, "mixed_bf16": 1, "mixed_bf16x3": 2, "mixed_tf32": 3}

# dram__bytes_read.sum + dram__bytes_write.sum per point of each stage's kernel, from one
# ncu capture at 384^3 (second correction of a solve; summarised under profiles/);
# traffic scales with points.  An entry must be removed when its kernel changes.  The
# x-inverse GEMM of a solve's first correction writes phi without reading it, so it has
# its own entry ("x_inverse_first").
MEASURED_TRAFFIC_PER_POINT = {
    ("residual", "mixed_bf16x3"): (921.222e6 + 213.402e6) / 384 ** 3,
    ("thomas", "mixed_bf16x3"): (226.622e6 + 179.088e6) / 384 ** 3,
    ("x_forward", "mixed_bf16x3"): (227.166e6 + 177.864e6) / 384 ** 3,
    ("y_forward", "mixed_bf16x3"): (227.126e6 + 174.007e6) / 384 ** 3,
    ("y_inverse", "mixed_bf16x3"): (227.184e6 + 178.220e6) / 384 ** 3,
    ("x_inverse", "mixed_bf16x3"): (681.377e6 + 389.205e6) / 384 ** 3,
    ("x_inverse_first", "mixed_bf16x3"): (227.420e6 + 388.045e6) / 384 ** 3,
}
DTYPE = {"fp64": "f64", "mixed_bf16": "bf16/f32/f64", "mixed_bf16x3": "bf16x3/f32/f64",
         "mixed_tf32": "tf32/f32/f64"}


def one_gpu_only(args) -> str | None:
    """Why this run is refused, or None: the solver runs on one GPU only."""
    world = _env_int("WORLD_SIZE", 1)
    if args.gpus != 1 or world != 1:
        return ("bench.py runs on one GPU only (got --gpus %d, WORLD_SIZE %d): the solve has no "
                "exchange step to shard, and its paired-CTA transform GEMMs share operand tiles by "
                "TMA multicast, which is kept to one-GPU runs" % (args.gpus, world))
    return None


def runs_reference_leg(rank: int) -> bool:
    """Under torchrun only rank 0 times the CPU oracle; the others exit 0."""
    return rank == 0


def run_ours(args):
    why = one_gpu_only(args)
    if why:
        print(why, file=sys.stderr, flush=True)
        return 2
    import torch

    local = 0
    torch.cuda.set_device(local)

    from paper_2603_09528_gb300 import build as _build
    _build.build()
    import paper_2603_09528_gb300 as tpt
    from paper_2603_09528_gb300 import _lib

    n, stretch = workload(args.size)
    grids = [tpt.grid_tanh(n[a], 1.0, stretch[a]) for a in range(3)]
    prec = PRECISIONS[args.precision]
    rtol = args.rtol if prec != 0 else 0.0
    refine = args.max_refine if args.max_refine is not None else (1 if prec == 0 else 8)
    plan = tpt.Plan(n, [g[0] for g in grids], [g[1] for g in grids], [(1, 1)] * 3,
                    xform=(tpt.GEMM, tpt.GEMM), alpha=0.0, beta=1.0, precision=prec,
                    rtol=rtol, max_refine=refine, device=local)
    f_host = rhs_host(n, grids)
    f_pin = torch.from_numpy(np.ascontiguousarray(f_host.ravel(order="F"))).pin_memory()
    f_dev = f_pin.to("cuda", non_blocking=False)
    phi = plan.new_field()
    work = plan.new_workspace()
    stream = torch.cuda.current_stream()

    tiles = None
    if prec != 0:
        if args.no_autotune:   # default tiles (for profiling runs: no tuning launches)
            tiles = plan.tiles()
        else:
            tiles = plan.autotune(work, stream=stream)   # transform GEMM column tiles per stage
    clocks = ClockSampler(local)
    clocks.start()
    # warm-up
    info = None
    for _ in range(args.warmup):
        _, info = plan.solve(f_dev, phi, work, stream=stream, want_info=True)
    torch.cuda.synchronize()

    clocks.mark(0)
    l0 = _lib.kernel_launches()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs[0].record(stream)
    infos = []
    for k in range(args.steps):
        _, inf = plan.solve(f_dev, phi, work, stream=stream, want_info=(rtol > 0 or prec != 0))
        infos.append(inf)
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    clocks.mark(1)
    l1 = _lib.kernel_launches()
    clk = clocks.stop()
    per = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    total_ms = evs[0].elapsed_time(evs[-1])
    value = args.steps / (total_ms / 1e3)
    npts = n[0] * n[1] * n[2]
    stages = None
    if prec != 0:
        # per-stage kernel times: the same solves again with CUDA events around
        # every stage (that mode synchronises once per correction, so it is kept
        # out of the timed region above)
        plan.set_stage_timing(True)
        tinfos = [plan.solve(f_dev, phi, work, stream=stream, want_info=True)[1] for _ in range(args.steps)]
        plan.set_stage_timing(False)
        ms = np.mean([i["ms_stage"] for i in tinfos], axis=0)
        its = float(np.mean([i["iters"] for i in tinfos]))
        stages = stage_rooflines(ms, its, n, prec)
        stages["per_solve_ms"] = {"input_conversion": float(ms[0]), "gauge_and_output": float(ms[7]),
                                  "stage_sum": float(np.sum(ms[0:8]))}

    # roofline of the dominant kernel
    if prec == 0:
        dom = dominant_kernel(plan, prec, n, f_dev, args.steps, stream)
    else:
        dom = max(stages["per_stage"], key=lambda d: d["ms_per_launch"] * d["launches_per_solve"])

    # end-to-end through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        phi_pin = torch.empty_like(f_pin).pin_memory()
        f2 = plan.new_field()
        plan.solve_host(f_pin, phi_pin, f2, phi, work, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            plan.solve_host(f_pin, phi_pin, f2, phi, work, stream=stream)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        one_at_a_time = {"value": args.steps / dt, "api": "tpt_solve_host, one call after another"}
        spec = dict(n=n, dxf=[g[0] for g in grids], dxc=[g[1] for g in grids], bc=[(1, 1)] * 3,
                    xform=(tpt.GEMM, tpt.GEMM), alpha=0.0, beta=1.0, precision=prec, rtol=rtol,
                    max_refine=refine)
        # a stream of requests long enough that filling and draining the
        # copy/solve pipeline, and a transient stall of the shared host link,
        # do not dominate the rate
        nreq = max(2 * args.steps, 40)
        srv = e2e_server(tpt, local, spec, f_pin, nreq, args.warmup, phi)
        dt_srv = srv.pop("seconds")
        e2e = {"value": nreq / dt_srv, "unit": "solves/s", "h2d_bytes_per_step": npts * 8,
               "d2h_bytes_per_step": npts * 8,
               "api": "tpt_server_submit / tpt_server_wait: consecutive solves from pinned host buffers, "
                      "each request's host-to-device copy, solve and device-to-host copy overlapping "
                      "those of its neighbours on %d slots" % srv["slots"],
               "server": srv, "one_call_at_a_time": one_at_a_time}

    # float64 path on the same workload, for the FP64-vs-mixed comparison
    fp64 = None
    if prec != 0 and not args.no_fp64:
        plan64 = tpt.Plan(n, [g[0] for g in grids], [g[1] for g in grids], [(1, 1)] * 3,
                          xform=(tpt.GEMM, tpt.GEMM), alpha=0.0, beta=1.0, precision=0,
                          max_refine=1, device=local)
        w64 = plan64.new_workspace()
        phi64 = plan64.new_field()
        _, i64 = plan64.solve(f_dev, phi64, w64, stream=stream, want_info=True)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 2
        a.record(stream)
        for _ in range(reps):
            plan64.solve(f_dev, phi64, w64, stream=stream, want_info=False)
        b.record(stream)
        torch.cuda.synchronize()
        ms64 = a.elapsed_time(b) / reps
        diff = (phi - phi64).abs().max().item() / phi64.abs().max().item()
        fp64 = {"solves_per_s": 1e3 / ms64, "ms_per_solve": ms64, "steps": reps,
                "rel_residual": i64["rel_residual"], "mixed_vs_fp64_max_rel_diff": diff}
        # the same tensor-core correction solves refined to float64 accuracy
        plan13 = tpt.Plan(n, [g[0] for g in grids], [g[1] for g in grids], [(1, 1)] * 3,
                          xform=(tpt.GEMM, tpt.GEMM), alpha=0.0, beta=1.0, precision=prec,
                          rtol=1e-13, max_refine=40, device=local)
        phi13 = plan13.new_field()
        _, i13 = plan13.solve(f_dev, phi13, work, stream=stream, want_info=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(args.steps):
            _, i13 = plan13.solve(f_dev, phi13, work, stream=stream, want_info=True)
        b.record(stream)
        torch.cuda.synchronize()
        ms13 = a.elapsed_time(b) / args.steps
        fp64["mixed_refined_to_1e-13"] = {
            "solves_per_s": 1e3 / ms13, "ms_per_solve": ms13, "iters": i13["iters"],
            "rel_residual": i13["rel_residual"],
            "max_rel_diff_vs_fp64": (phi13 - phi64).abs().max().item() / phi64.abs().max().item()}
        del plan13, phi13
        # float64-accurate transforms by the Ozaki scheme on the bf16 tensor cores
        planoz = tpt.Plan(n, [g[0] for g in grids], [g[1] for g in grids], [(1, 1)] * 3,
                          xform=(tpt.GEMM, tpt.GEMM), alpha=0.0, beta=1.0, precision=4, max_refine=1,
                          device=local)
        woz, phioz = planoz.new_workspace(), planoz.new_field()
        _, ioz = planoz.solve(f_dev, phioz, woz, stream=stream, want_info=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            planoz.solve(f_dev, phioz, woz, stream=stream, want_info=False)
        b.record(stream)
        torch.cuda.synchronize()
        msoz = a.elapsed_time(b) / reps
        fp64["ozaki"] = {
            "solves_per_s": 1e3 / msoz, "ms_per_solve": msoz, "steps": reps, "rel_residual": ioz["rel_residual"],
            "speedup_vs_fp64": ms64 / msoz,
            "max_rel_diff_vs_fp64": (phioz - phi64).abs().max().item() / phi64.abs().max().item(),
            "scheme": "7 bf16 slices of 6 bits per operand row, levels 2..8 exact in float32, float64 sum"}
        del planoz, woz, phioz
        del w64, phi64, plan64
        torch.cuda.empty_cache()

    projection = None
    if not args.no_projection and prec != 0:
        projection = projection_leg(tpt, plan, n, stream, args.steps)

    fft = None
    if not args.no_fft:
        fft = fft_leg(tpt, tuple(args.fft_shape) if args.fft_shape else n, stream, args.steps)

    batch = None
    if not args.no_batch:
        batch = {"mixed": batch_leg(tpt, local, stream, prec if prec != 0 else 2, args.steps)}
        if not args.no_fp64:
            batch["fp64"] = batch_leg(tpt, local, stream, 0, args.steps)

    serving = None
    if not args.no_serving:
        serving = {"mixed": serving_leg(tpt, local, prec if prec != 0 else 2, args.serve_requests,
                                        args.serve_warmup)}
        serving["same_shape_bursts"] = [merge_leg(tpt, local, count=96, n=(64, 64, 64), slots=2),
                                        merge_leg(tpt, local, count=64, n=(96, 96, 96), slots=4)]
        if not args.no_fp64:
            serving["fp64"] = serving_leg(tpt, local, 0, args.serve_requests_fp64, 10)

    cpu = None
    if not args.no_cpu_baseline:
        nslab = max(1, min(n[2], args.cpu_slabs))
        cpu = cpu_baseline_record(n, args.size, nslab, cpu_sample(n, nslab))

    last = next((i for i in reversed(infos) if i), info)
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[args.precision], "data": "synthetic",
        "config": {"workload": workload_name(args.size),
                   "size": list(n), "stretch": list(stretch), "precision": args.precision,
                   "rtol": rtol, "max_refine": refine, "parallelism": "single GPU",
                   "gemm_tiles": tiles,
                   "l2": "inputs larger than L2 (%.2f GB field)" % (npts * 8 / 1e9)},
        "gpts_per_s": value * npts / 1e9,
        "latency_ms": {"p50": float(np.percentile(per, 50)), "p99": float(np.percentile(per, 99)),
                       "mean20fastest": float(np.mean(sorted(per)[:20]))},
        "solve_info": {k: v for k, v in (last or {}).items() if k != "ms_stage"},
        "stages": stages,
        "fp64": fp64,
        "projection": projection,
        "fft": fft,
        "batch": batch,
        "serving": serving,
        "gpu_launches": l1 - l0,
        "roofline": dom,
        "clocks": clk,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    print(json.dumps(out), flush=True)
    return 0


def batch_leg(tpt, device, stream, prec, steps, count=96, seed=5, nstreams=8):
    """Batched uneven instances (sizes from {64^3, 96x128x160, 128^3,
    192x192x96, 256^3}, half Poisson / half Helmholtz with dt*nu in (0, 1e-2],
    stretching U[1, 3] per direction, Neumann walls): every instance solved in
    one CUDA graph replay.  Mixed instances first get their correction count
    from one adaptive solve each (rtol 1e-10) and their GEMM tiles from the
    autotuner.  Right-hand sides are seeded uniform[-1, 1] drawn on the device."""
    import torch
    import seeded_inputs as S
    inst = S.batch_instances(count, seed)
    specs = []
    t0 = time.perf_counter()
    for it in inst:
        n = it["n"]
        grids = [tpt.grid_tanh(n[a], 1.0, it["stretch"][a]) for a in range(3)]
        specs.append(dict(n=n, dxf=[g[0] for g in grids], dxc=[g[1] for g in grids], bc=[(1, 1)] * 3,
                          xform=(tpt.GEMM, tpt.GEMM), alpha=it["alpha"], beta=it["beta"], precision=prec,
                          rtol=1e-10 if prec != 0 else 0.0, max_refine=1 if prec == 0 else 8))
    b = tpt.Batch(specs, nstreams=nstreams, device=device)
    t_setup = time.perf_counter() - t0
    gen = torch.Generator(device="cuda:%d" % device)
    fs, phis = [], []
    for i, it in enumerate(inst):
        gen.manual_seed(it["seed"])
        npts = it["n"][0] * it["n"][1] * it["n"][2]
        fs.append(torch.rand(npts, generator=gen, dtype=torch.float64, device="cuda:%d" % device) * 2 - 1)
        phis.append(torch.empty_like(fs[-1]))
    work = b.new_workspace()
    t0 = time.perf_counter()
    # the corrections each instance needs, no spare: the stopping test still
    # runs on the device, and an instance that misses rtol reports it
    corrections = b.calibrate(fs, phis, work, rtol=1e-10, spare=0) if prec != 0 else [2] * count
    t_cal = time.perf_counter() - t0
    t0 = time.perf_counter()
    tiles = b.autotune(work, stream) if prec != 0 else None
    t_tune = time.perf_counter() - t0
    reps = max(2, steps) if prec != 0 else 2

    def timed(work):
        t0 = time.perf_counter()
        b.solve(fs, phis, work, stream=stream)        # eager run + graph capture
        t_cap = time.perf_counter() - t0
        for _ in range(2):
            b.solve(fs, phis, work, stream=stream, want_info=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            b.solve(fs, phis, work, stream=stream, want_info=False)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, t_cap

    grouped = b.grouped
    streams_mode = None
    if grouped:
        # the capture streams on the same instances, for comparison
        b.set_grouped(False)
        ws = b.new_workspace()
        ms_s, _ = timed(ws)
        streams_mode = {"ms_per_batch": ms_s, "gpts_per_s": sum(it["n"][0] * it["n"][1] * it["n"][2]
                                                                for it in inst) / (ms_s / 1e3) / 1e9,
                        "launches_per_replay": b.launches_per_replay(), "nstreams": nstreams}
        del ws
        b.set_grouped(True)
        work = b.new_workspace()
    ms, t_capture = timed(work)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = b.solve(fs, phis, work, stream=stream)
    # the same instances one after another on one stream, without the graph
    for p, inf in zip(b.plans, infos):
        p.set_refinement(0.0, inf["iters"] - 1)
    e0.record(stream)
    for p, f, phi in zip(b.plans, fs, phis):
        p.solve(f, phi, work, stream=stream, want_info=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    pts = sum(it["n"][0] * it["n"][1] * it["n"][2] for it in inst)
    res = [i["rel_residual"] for i in infos]
    out = {"instances": count, "points": pts, "precision": {0: "fp64", 1: "mixed_bf16", 2: "mixed_bf16x3",
                                                              3: "mixed_tf32"}[prec],
           "mode": "grouped launches (one kernel per stage over all instances)" if grouped
           else "capture streams", "nstreams": None if grouped else nstreams, "ms_per_batch": ms, "steps": reps,
           "capture_streams_mode": streams_mode,
           "solves_per_s": count * 1e3 / ms, "gpts_per_s": pts / (ms / 1e3) / 1e9,
           "sequential_ms": ms_seq, "graph_speedup_vs_sequential": ms_seq / ms,
           "launches_per_replay": b.launches_per_replay(), "graph_launches_per_batch": 1,
           "corrections": {"min": min(corrections), "max": max(corrections),
                           "mean": float(np.mean(corrections))},
           "max_rel_residual": max(res), "not_ok": sum(1 for i in infos if i["status"] != 0),
           "setup_s": {"plans": t_setup, "calibration": t_cal, "autotune": t_tune,
                       "first_call_with_capture": t_capture}}
    if tiles is not None:
        hist = {}
        for t in tiles:
            for st, w in zip(("x_fwd", "y_fwd", "y_inv", "x_inv"), t):
                hist.setdefault(st, {}).setdefault(str(w), 0)
                hist[st][str(w)] += 1
        out["autotuned_tiles"] = hist
    b.close()
    del fs, phis, work
    torch.cuda.empty_cache()
    return out


def serving_leg(tpt, device, prec, count, warmup, rate_hz=200.0, slots=4, stretch_step=0.25):
    """Open-loop serving (Poisson arrivals at rate_hz; sizes per dimension
    uniform over {64, 96, ..., 512}; 70% Poisson / 30% Helmholtz; stretch
    factors on [1, 3] in steps of stretch_step) through the continuous-batching
    server.  Every request's right-hand side is the first N_x N_y N_z values of
    one seeded pinned host field and its solution is copied back into one of a
    ring of pinned host buffers (contents are not kept: timing only).  The
    first `warmup` requests fill the eigenbasis cache and are not counted;
    latency = completion - submission on the server's clock."""
    import threading
    import torch
    import seeded_inputs as S
    reqs = S.serving_requests(warmup + count, rate_hz=rate_hz, seed=6, stretch_step=stretch_step)
    nmax = max(r["n"][0] * r["n"][1] * r["n"][2] for r in reqs)
    gen = torch.Generator(device="cuda:%d" % device)
    gen.manual_seed(6)
    f_host = (torch.rand(nmax, generator=gen, dtype=torch.float64, device="cuda:%d" % device) * 2 - 1).cpu()
    f_host = f_host.pin_memory()
    ring = [torch.empty(nmax, dtype=torch.float64).pin_memory() for _ in range(slots + 4)]
    srv = tpt.Server(device=device, slots=slots, setup_threads=min(8, max(2, (os.cpu_count() or 4) // 2)),
                     memory_budget=96 << 30, cache_budget=16 << 30)
    grids = {}

    def spec(r):
        gs = []
        for a in range(3):
            key = (r["n"][a], r["stretch"][a])
            if key not in grids:
                grids[key] = tpt.grid_tanh(r["n"][a], 1.0, r["stretch"][a])
            gs.append(grids[key])
        mixed = prec != 0
        return dict(n=r["n"], dxf=[g[0] for g in gs], dxc=[g[1] for g in gs], bc=[(1, 1)] * 3,
                    xform=(tpt.GEMM, tpt.GEMM), alpha=r["alpha"], beta=r["beta"], precision=prec,
                    rtol=1e-10 if mixed else 0.0, max_refine=30 if mixed else 1)

    specs = [spec(r) for r in reqs]
    # the mesh library is known ahead of traffic: build every direction's
    # eigenbasis once (R16), as a deployment would at start-up
    t0w = time.perf_counter()
    seen = set()
    for r in reqs:
        for a in range(2):
            key = (r["n"][a], r["stretch"][a])
            if key in seen:
                continue
            seen.add(key)
            g = grids[key]
            small = tpt.grid_tanh(8, 1.0, 1.0)
            srv.warm(n=(key[0], 8, 8), dxf=[g[0], small[0], small[0]], dxc=[g[1], small[1], small[1]],
                     bc=[(1, 1)] * 3, xform=(tpt.GEMM, tpt.GEMM), alpha=1.0, beta=-1e-3, precision=prec,
                     rtol=0.0, max_refine=1)
    t_warm = time.perf_counter() - t0w
    tickets = [None] * len(reqs)
    results = [None] * len(reqs)
    submitted = threading.Event()

    def collector():
        for i in range(len(reqs)):
            while tickets[i] is None:
                time.sleep(0.0005)
            results[i] = srv.wait(tickets[i])

    th = threading.Thread(target=collector, daemon=True)
    th.start()
    t0 = time.perf_counter()
    for i, r in enumerate(reqs):
        delay = r["t_arrival"] - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        tickets[i] = srv.submit(f_host, ring[i % len(ring)], **specs[i])
    submitted.set()
    th.join()
    st = srv.stats()
    srv.close()
    meas = results[warmup:]
    lat = np.array([(x["t_done"] - x["t_submit"]) * 1e3 for x in meas])
    plan_ms = np.array([(x["t_planned"] - x["t_submit"]) * 1e3 for x in meas])
    queue_ms = np.array([(x["t_admit"] - x["t_planned"]) * 1e3 for x in meas])
    run_ms = np.array([(x["t_done"] - x["t_admit"]) * 1e3 for x in meas])
    span = max(x["t_done"] for x in meas) - min(x["t_submit"] for x in meas)
    pts = sum(r["n"][0] * r["n"][1] * r["n"][2] for r in reqs[warmup:])
    bad = sum(1 for x in meas if x["status"] != 0)
    statuses, failures = {}, []
    for x in results:
        if x["status"] != 0:
            statuses[str(x["status"])] = statuses.get(str(x["status"]), 0) + 1
            failures.append({"status": x["status"], "step": x.get("failed_step"),
                             "cuda_error": x.get("cuda_error_name")})
    return {"precision": {0: "fp64", 1: "mixed_bf16", 2: "mixed_bf16x3", 3: "mixed_tf32"}[prec],
            "requests": count, "warmup_requests": warmup, "offered_rate_hz": rate_hz,
            "slots": slots, "stretch_step": stretch_step,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "mean": float(lat.mean()), "max": float(lat.max())},
            "phase_ms_p50": {"plan": float(np.median(plan_ms)), "queue": float(np.median(queue_ms)),
                             "h2d_solve_d2h": float(np.median(run_ms))},
            "solves_per_s": count / span, "gpts_per_s": pts / span / 1e9,
            "same_shape_batching": {"merge": 8, "merged_fraction": float(np.mean([x.get("merged", 1) > 1
                                                                                 for x in meas])),
                                    "max_merged": int(max(x.get("merged", 1) for x in meas))},
            "failed": bad, "failed_statuses": statuses, "failures": failures[:8], "warm_s": t_warm, "warmed_plans": len(seen),
            "max_rel_residual": float(max(x["rel_residual"] for x in meas)),
            "cache": {"hits": int(st["cache_hits"]), "misses": int(st["cache_misses"]),
                      "device_bytes": int(st["cache_bytes"])},
            "peak_inflight": int(st["peak_inflight"]), "peak_device_bytes": int(st["peak_bytes"])}


def merge_leg(tpt, device, count=64, n=(96, 96, 96), slots=4):
    """Same-shape batching: `count` requests of one grid size (split bf16
    Helmholtz, rtol 1e-10, stretching varied per request so each has its own
    eigenbases) submitted at once, served with merging off and with up to 8
    requests solved together; solves/s from the first submission to the last
    completion (median of three bursts), and p50/p99 of the request latency
    over the three."""
    import torch
    npts = n[0] * n[1] * n[2]
    f = (torch.rand(npts, dtype=torch.float64) * 2 - 1).pin_memory()
    outs = [torch.empty(npts, dtype=torch.float64).pin_memory() for _ in range(count)]
    specs = []
    for i in range(count):
        st = (1.0 + 0.25 * (i % 5), 1.25 + 0.25 * (i % 4), 1.5 + 0.25 * (i % 3))
        gs = [tpt.grid_tanh(n[a], 1.0, st[a]) for a in range(3)]
        specs.append(dict(n=n, dxf=[g[0] for g in gs], dxc=[g[1] for g in gs], bc=[(1, 1)] * 3,
                          xform=(tpt.GEMM, tpt.GEMM), alpha=1.0, beta=-5e-4, precision=2, rtol=1e-10,
                          max_refine=30))
    out = {"requests": count, "grid": list(n), "slots": slots, "bursts": 3}
    for merge in (1, 8):
        srv = tpt.Server(device=device, slots=slots, setup_threads=4, memory_budget=32 << 30,
                         cache_budget=4 << 30, merge=merge)
        rates, lat, res = [], [], []
        try:
            for sp in specs:
                srv.warm(**sp)
            for t in [srv.submit(f, outs[i], **specs[i]) for i in range(8)]:   # warm-up
                srv.wait(t, timeout=300.0)
            # three bursts: one straggling request decides a whole ~20 ms burst,
            # so the median burst is reported beside each burst's rate
            for _ in range(3):
                t0 = time.perf_counter()
                tickets = [srv.submit(f, outs[i], **specs[i]) for i in range(count)]
                rb = [srv.wait(t, timeout=300.0) for t in tickets]
                rates.append(count / (time.perf_counter() - t0))
                lat += [(r["t_done"] - r["t_submit"]) * 1e3 for r in rb]
                res += rb
        finally:
            srv.close()
        lat = np.array(lat)
        out["merge%d" % merge] = {"solves_per_s": float(np.median(rates)), "bursts_solves_per_s": rates,
                                  "p50_ms": float(np.percentile(lat, 50)),
                                  "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
                                  "mean_merged": float(np.mean([r["merged"] for r in res])),
                                  "failed": sum(1 for r in res if r["status"] != 0),
                                  "max_rel_residual": float(max(r["rel_residual"] for r in res))}
    return out


def fft_leg(tpt, n, stream, steps):
    """float64 path with Fourier-based x and y transforms (Sec. 2.2.1, uniform
    grids): uniform x and y (Neumann walls: DCT-II / DCT-III; periodic: real
    DFT), z stretched 2.0 and solved by Thomas, Helmholtz (1, -5e-4).  Each
    transform is timed alone with CUDA events (seeded uniform[0, 1) input),
    then the whole solve.  Algorithmic work per point and transform: 16 bytes
    (one float64 read, one write) and 2.5 log2(N) + 6 float64 flops (one radix-2
    complex FFT of length N for two real lines, plus the pre/post rotation and
    the separation of the two lines' spectra)."""
    import torch
    out = {}
    npts = n[0] * n[1] * n[2]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(11)
    for kind, bc in (("neumann_dct", (1, 1)), ("periodic_dft", (0, 0))):
        if any(n[a] & (n[a] - 1) for a in (0, 1)):
            return None   # power-of-two x and y only
        grids = [tpt.grid_tanh(n[a], 1.0, 0.0 if a < 2 else 2.0) for a in range(3)]
        plan = tpt.Plan(n, [g[0] for g in grids], [g[1] for g in grids], [bc, bc, (1, 1)],
                        xform=(tpt.FFT, tpt.FFT), alpha=1.0, beta=-5e-4, precision=0, max_refine=1)
        f = torch.rand(npts, generator=gen, dtype=torch.float64, device="cuda")
        y = plan.new_field()
        rec = {}
        for d in (0, 1):
            N = n[d]
            flops = npts * (2.5 * np.log2(N) + 6.0)
            for inv in (False, True):
                for _ in range(2):
                    plan.transform(f, d, inv, out=y, stream=stream)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                reps = max(3, steps)
                e0.record(stream)
                for _ in range(reps):
                    plan.transform(f, d, inv, out=y, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                rec["%s_%s" % ("xy"[d], "inverse" if inv else "forward")] = {
                    "ms": ms, "gb_per_s": 16.0 * npts / (ms / 1e3) / 1e9,
                    "fp64_gflop_per_s": flops / (ms / 1e3) / 1e9}
        phi, work = plan.new_field(), plan.new_workspace()
        plan.solve(f, phi, work, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = max(2, min(steps, 3))
        e0.record(stream)
        for _ in range(reps):
            _, info = plan.solve(f, phi, work, stream=stream, want_info=True)
        e1.record(stream)
        torch.cuda.synchronize()
        rec["solve"] = {"ms": e0.elapsed_time(e1) / reps, "iters": info["iters"],
                        "rel_residual": info["rel_residual"]}
        rec["mixed"] = fft_mixed_leg(tpt, n, grids, bc, f, stream, steps)
        out[kind] = rec
        del plan, f, y, phi, work
        torch.cuda.empty_cache()
    out["workload"] = "helmholtz_%dx%dx%d_uniform_xy_tanh2.0_z_fp64_fft" % tuple(n)
    return out


def fft_mixed_leg(tpt, n, grids, bc, f, stream, steps):
    """The same Helmholtz problem solved by the split-bf16 refined path (rtol
    1e-10) with float32 FFT/DCT transforms in x and y, and with the tensor-core
    eigenbasis GEMMs for comparison: solve time and, from the stage timing
    pass, each Fourier stage's time per launch against the HBM peak.
    Algorithmic bytes per point: 8 for x forward (split-bf16 rows in and out),
    y forward (split bf16 in, float32 out) and y inverse; x inverse 4 in plus
    the float-pair phi (8 written in the first correction, 16 read and written
    in the later ones)."""
    import torch
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    npts = n[0] * n[1] * n[2]
    res = {}
    for name, xf in (("fft", (tpt.FFT, tpt.FFT)), ("gemm", (tpt.GEMM, tpt.GEMM))):
        plan = tpt.Plan(n, [g[0] for g in grids], [g[1] for g in grids], [bc, bc, (1, 1)], xform=xf,
                        alpha=1.0, beta=-5e-4, precision=PRECISIONS["mixed_bf16x3"], rtol=1e-10, max_refine=8)
        phi, work = plan.new_field(), plan.new_workspace()
        if name == "gemm":
            plan.autotune(work, stream=stream)
        for _ in range(3):
            plan.solve(f, phi, work, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = max(3, steps)
        e0.record(stream)
        for _ in range(reps):
            _, info = plan.solve(f, phi, work, stream=stream, want_info=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        plan.set_stage_timing(True)
        ti = [plan.solve(f, phi, work, stream=stream, want_info=True)[1] for _ in range(2)]
        plan.set_stage_timing(False)
        st = np.mean([t["ms_stage"] for t in ti], axis=0)
        its = float(np.mean([t["iters"] for t in ti]))
        r = {"ms": ms, "solves_per_s": 1e3 / ms, "iters": info["iters"], "rel_residual": info["rel_residual"]}
        if name == "fft":
            stages = {}
            xinv_bytes = 4.0 + (8.0 + 16.0 * (its - 1.0)) / its
            for key, i, bpp in (("x_forward", 1, 8.0), ("y_forward", 2, 8.0), ("y_inverse", 4, 8.0),
                                ("x_inverse", 5, xinv_bytes)):
                per = float(st[i]) / its
                gbs = bpp * npts / (per / 1e3) / 1e9
                stages[key] = {"ms_per_launch": per, "bytes_per_point": bpp, "achieved_gbs": gbs,
                               "frac_of_hbm": gbs / hbm}
            r["stages"] = stages
        res[name] = r
        del plan, phi, work
        torch.cuda.empty_cache()
    res["precision"] = "mixed_bf16x3, float32 FFT/DCT in x and y (gemm: tensor-core eigenbasis GEMMs)"
    return res


def projection_leg(tpt, plan, n, stream, steps):
    """Pressure projection (Sec. 2.1) on the benchmark grid: D u* / g, the
    refined Poisson solve, u -= g G Phi, with seeded uniform[-1, 1] face
    velocities (zero normal velocity on the walls).  Each step restores the
    starting velocity outside its timed region (CUDA events around
    tpt_project only)."""
    import torch
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    shapes = [(n[0] + 1, n[1], n[2]), (n[0], n[1] + 1, n[2]), (n[0], n[1], n[2] + 1)]
    start = []
    for ax, shp in enumerate(shapes):
        t = torch.rand(shp[::-1], generator=gen, dtype=torch.float64, device="cuda") * 2 - 1   # (z, y, x)
        idx = [slice(None)] * 3
        idx[2 - ax] = 0
        t[tuple(idx)] = 0.0
        idx[2 - ax] = -1
        t[tuple(idx)] = 0.0
        start.append(t.reshape(-1))
    work = [t.clone() for t in start]
    ws = plan.project_workspace()
    phi = plan.new_field()
    gdt = 0.125
    for _ in range(2):
        for w_, s_ in zip(work, start):
            w_.copy_(s_)
        plan.project(*work, gdt, phi=phi, work=ws, stream=stream)
    times = []
    for _ in range(max(3, steps)):
        for w_, s_ in zip(work, start):
            w_.copy_(s_)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        _, info = plan.project(*work, gdt, phi=phi, work=ws, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    npts = n[0] * n[1] * n[2]
    ms = float(np.median(times))
    del work, start, ws, phi
    torch.cuda.empty_cache()
    return {"workload": "projection_%dx%dx%d_tanh1.5-2.0-2.5_neumann" % n, "ms_per_projection": ms,
            "projections_per_s": 1e3 / ms, "gpts_per_s": npts / (ms / 1e3) / 1e9, "steps": len(times),
            "solve_iters": info["iters"], "rel_residual": info["rel_residual"],
            "bytes_outside_solve_per_point": 32 + 56}


# The float-pair residual of the singular headline problem is bound by the
# float32 datapath (ncu: FMA pipe 66 % busy, math-pipe throttle the largest
# stall), not by HBM.  Its float32 operations per point, counted from the
# kernel's arithmetic: 4.5 exact face differences (8 each: TwoSum and the lo
# parts; z 1, y 2, x 1.5 as the face between the two points of a lane is
# differenced once), six exact coefficient products with their TwoSum
# accumulation (12 each), the compatibility shift of f (8), the final hi + lo
# (1) and the r^2 sum (1).  Peak: 152 SMs x 128 float32 lanes x 2.070 GHz
# (unit counts and the maximum SM clock), one operation per lane and clock.
RESIDUAL_F32_OPS = 36 + 6 * 12 + 8 + 1 + 1
F32_LANE_TOPS = 152 * 128 * 2.070e9 / 1e12


def stage_rooflines(ms, iters, n, prec):
    """Per-stage achieved rates from the solve's own CUDA-event stage timings.
    Algorithmic work per point and launch: transforms 2*N_alpha flop per
    product (3 products for split bf16) and their operand/result bytes;
    Thomas and residual their field bytes."""
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    tflops = peaks.get("bf16_tflops", 1900.0)
    if prec == 3:
        tflops = tflops / 2.0          # tf32 dense rate is half the bf16 rate
    npts = float(n[0] * n[1] * n[2])
    eb = {1: 2, 2: 4, 3: 4}[prec]      # bytes per stored intermediate value
    prods = 3 if prec == 2 else 1
    names = ["prepare", "x_forward", "y_forward", "thomas", "y_inverse", "x_inverse", "residual"]
    out = []
    for i, nm in enumerate(names[1:], start=1):
        per_launch = ms[i] / max(iters, 1)
        if nm in ("x_forward", "y_forward", "y_inverse", "x_inverse"):
            na = n[0] if nm.startswith("x") else n[1]
            flops = 2.0 * na * npts * prods
            # the x inverse updates the float-pair phi: read and write (16 B/pt), except
            # in a solve's first correction, which only writes it (8 B/pt)
            first = 1.0 / max(iters, 1)
            byts = npts * (eb + (16.0 - 8.0 * first if nm == "x_inverse" else eb))
            t_tensor = flops / (tflops * 1e12)
            t_hbm = byts / (hbm * 1e9)
            if t_tensor >= t_hbm:
                d = {"bound": "tensor", "achieved": flops / (per_launch / 1e3) / 1e12, "peak": tflops,
                     "unit": "TFLOP/s"}
            else:
                d = {"bound": "hbm", "achieved": byts / (per_launch / 1e3) / 1e9, "peak": hbm, "unit": "GB/s"}
            d["flops_per_launch"] = flops
        else:
            byts = npts * (2 * eb if nm == "thomas" else 8 + 8 + eb)
            d = {"bound": "hbm", "achieved": byts / (per_launch / 1e3) / 1e9, "peak": hbm, "unit": "GB/s"}
        d.update({"kernel": nm, "ms_per_launch": per_launch, "launches_per_solve": iters,
                  "bytes_per_launch": byts, "traffic": None})
        d["frac"] = d["achieved"] / d["peak"]
        if nm == "residual":
            # the unit that bounds it: the float32 datapath (see RESIDUAL_F32_OPS)
            ops = RESIDUAL_F32_OPS * npts
            achieved = ops / (per_launch / 1e3) / 1e12
            d["alu"] = {"bound": "alu", "ops_per_point": RESIDUAL_F32_OPS, "achieved": achieved,
                        "peak": F32_LANE_TOPS, "unit": "Tops/s (float32 lane operations)",
                        "frac": achieved / F32_LANE_TOPS}
        out.append(d)
    fmt = {1: "mixed_bf16", 2: "mixed_bf16x3", 3: "mixed_tf32"}[prec]
    for d in out:
        key = (d["kernel"], fmt)
        if d["kernel"] == "x_inverse":   # average launch: one first correction per solve
            k1 = ("x_inverse_first", fmt)
            if key in MEASURED_TRAFFIC_PER_POINT and k1 in MEASURED_TRAFFIC_PER_POINT:
                first = 1.0 / max(iters, 1)
                d["traffic"] = npts * (first * MEASURED_TRAFFIC_PER_POINT[k1] +
                                       (1.0 - first) * MEASURED_TRAFFIC_PER_POINT[key])
        elif key in MEASURED_TRAFFIC_PER_POINT:
            d["traffic"] = MEASURED_TRAFFIC_PER_POINT[key] * npts
    return {"per_stage": out, "iters": iters, "peak_source": "MEASURED_PEAKS.json (burst)"}


def e2e_server(tpt, device, spec, f_pin, steps, warmup, phi_ref, slots=3):
    """End to end through the serving API: `steps` solves of the headline
    workload submitted back to back with pinned host buffers (f read from
    host memory, phi written back to host memory by every request), timed from
    the first submission to the last completion; the server overlaps each
    request's copies with its neighbours' solves.  The last result is checked
    against the solve of the same right-hand side on the device."""
    import torch
    npts = f_pin.numel()
    ring = [torch.empty(npts, dtype=torch.float64).pin_memory() for _ in range(2 * slots + 2)]
    srv = tpt.Server(device=device, slots=slots, setup_threads=2, memory_budget=64 << 30,
                     cache_budget=8 << 30)
    try:
        srv.warm(**spec)
        for t in [srv.submit(f_pin, ring[i % len(ring)], **spec) for i in range(warmup)]:
            r = srv.wait(t, timeout=300.0)
            if r is None or r["status"] != 0:
                raise RuntimeError("e2e warm-up request failed: %r" % (r,))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tickets = [srv.submit(f_pin, ring[i % len(ring)], **spec) for i in range(steps)]
        res = [srv.wait(t, timeout=300.0) for t in tickets]
        seconds = time.perf_counter() - t0
    finally:
        srv.close()
    bad = [r for r in res if r is None or r["status"] != 0]
    if bad:
        raise RuntimeError("e2e request failed: %r" % (bad[0],))
    ref = phi_ref.cpu()
    last = ring[(steps - 1) % len(ring)]
    diff = float((last - ref).abs().max() / ref.abs().max())
    t0s = res[0]["t_submit"]
    done = sorted(r["t_done"] for r in res)
    gaps = [1e3 * (b - a) for a, b in zip(done, done[1:])]
    return {"seconds": seconds, "slots": slots, "requests": steps,
            "completion_gap_ms": {"median": float(np.median(gaps)), "max": float(max(gaps))} if gaps else None,
            # one completion per median gap once the slots are busy (the timed
            # region above also holds the pipeline fill of the first requests)
            "steady_state_solves_per_s": 1e3 / float(np.median(gaps)) if gaps else None,
            "max_rel_residual": max(r["rel_residual"] for r in res),
            "max_rel_diff_vs_device_solve": diff,
            "timeline_ms": {k: [round((r[key] - t0s) * 1e3, 2) for r in res]
                            for k, key in (("planned", "t_planned"), ("admitted", "t_admit"),
                                           ("copied", "t_copied"), ("solved", "t_solved"), ("done", "t_done"))}}


def dominant_kernel(plan, prec, n, f_dev, steps, stream):
    """Times the solve's dominant kernel alone (same kernel and launch shape as
    inside tpt_solve) with CUDA events on the launching stream."""
    import torch
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    out = plan.new_field()
    reps = max(3, steps)
    plan.transform(f_dev, 0, False, out=out, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        plan.transform(f_dev, 0, False, out=out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    flops = 2.0 * n[0] * n[0] * n[1] * n[2]
    achieved = flops / (ms / 1e3) / 1e12
    if prec == 0:
        peak = 1.25   # GB300 float64 rate in TFLOP/s, nominal (an FMA counts two flops)
        return {"kernel": "dgemm_cm_kernel (x forward transform)", "bound": "alu",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": "nominal GB300 float64 rate (MEASURED_PEAKS.json has no float64 entry)",
                "traffic": None, "ms_per_launch": ms, "flops_per_launch": flops}
    peak = peaks.get("bf16_tflops", 1900.0)
    return {"kernel": "x forward transform", "bound": "tensor", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None, "ms_per_launch": ms}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed_bf16x3", choices=list(PRECISIONS))
    ap.add_argument("--no-fp64", action="store_true", help="skip the float64-path comparison leg")
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--rtol", type=float, default=1e-10)
    ap.add_argument("--max-refine", type=int, default=None)
    ap.add_argument("--cpu-slabs", type=int, default=128)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fft", action="store_true", help="skip the float64 FFT/DCT-transform leg")
    ap.add_argument("--fft-shape", type=int, nargs=3, default=None, metavar=("NX", "NY", "NZ"),
                    help="grid of the FFT/DCT leg (power-of-two NX, NY; default: the headline grid)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched uneven-instances leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the open-loop serving leg")
    ap.add_argument("--no-projection", action="store_true", help="skip the pressure-projection leg")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default GEMM tiles of the headline plan (profiling runs)")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-warmup", type=int, default=200)
    ap.add_argument("--serve-requests-fp64", type=int, default=40)
    ap.add_argument("--cpu-sample-only", type=int, default=0, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_sample_only:   # child of cpu_single_thread: seconds per solve, no GPU
        print(cpu_sample(workload(args.size)[0], args.cpu_sample_only))
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
