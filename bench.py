"""Benchmark of the fast QMC product B = Y·A on GB300.

Default workload (gauss-65537): rank-1 lattice with N = 65537, s = t = 4096,
Φ^{-1} map, Korobov generating vector, A = upper Cholesky factor of
min(i,k)/s (Section 3.1 / Section 4, Experiment 1 shape), FP32 path.

One step = one forward product (scatter-add, FFT, spectral product,
inverse FFT, un-permute) over the whole batch of t columns.  Prints one JSON
line.  `--impl reference` times the FP64 CPU oracle on a bounded sample of
the same workload instead.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1501_06286_gb300 import workloads  # noqa: E402

METRIC = "Y·A outputs/s (N·t/s), FFT vs dense GEMM on 1 GB300 at max rel err ≤1e-5"
UNIT = "outputs/s"


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def _make_workload(name: str, rank: int, grid: int | None = None):
    # grid: a smaller node grid for the field workloads (profiling captures)
    if name == "gauss-65537":
        return workloads.gauss_65537(seed=1)
    if name == "field-786433":
        w = workloads.field_786433(seed=2, **({"grid": grid} if grid else {}))
        if grid:
            w.name = f"field-786433-grid{grid}"
        return w
    if name == "f2-65536":
        w = workloads.f2_65536(seed=4, **({"grid": grid} if grid else {}))
        if grid:
            w.name = f"f2-65536-grid{grid}"
        return w
    if name == "lattice-257":
        return workloads.lattice_257(seed=0)
    if name == "batch-64":
        return workloads.batch_64(seed=3)[0]
    # Experiments 2 and 3 of the paper at M = s = 2N (N = 4001): the assembly
    # b = a_0 + Y·a, and the log-normal field exp(2 + Y·Ψ)
    if name == "fe-uniform-4001":
        return workloads.fe_workload("uniform", 4001, M=8002, s=8002)
    if name == "fe-lognormal-4001":
        return workloads.fe_workload("lognormal", 4001, M=8002, s=8002)
    raise SystemExit(f"unknown workload {name}")


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self._proc = None
        self._thr = None

    def _reader(self):
        for line in self._proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __enter__(self):
        try:
            self._proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._thr = threading.Thread(target=self._reader, daemon=True)
            self._thr.start()
            time.sleep(0.3)  # first sample before the timed work starts
        except Exception:
            self._proc = None
        return self

    def __exit__(self, *exc):
        if self._proc is not None:
            time.sleep(0.1)
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()
            self._thr.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = [num(r[0]) for r in self.rows]
        mx = [num(r[1]) for r in self.rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for nm, v in zip(names, r[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(self.rows),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
def _oracle_pointset(w):
    from oracle import f2, points
    if w.kind == "prime":
        return points.PointSet("prime", w.N, w.gen, w.map, w.row0)
    m = w.extra["m"]
    P = f2.smallest_primitive(m)
    q = [f2.x_power_fast(int(e), P) for e in w.gen]
    return points.PointSet("f2", w.N, q, w.map, w.row0, P=P)


def oracle_rate(w, seconds: float):
    """FP64 oracle outputs/s on consecutive row blocks of the workload."""
    from oracle import products
    ps = _oracle_pointset(w)
    A = w.A.astype(np.float64)
    block = 256
    rows = 0
    t0 = time.perf_counter()
    r0 = 0
    while True:
        r1 = min(ps.out_rows, r0 + block)
        products.matmul_rows(ps, A, np.arange(r0, r1))
        rows += r1 - r0
        r0 = r1 % ps.out_rows
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return rows * w.t / el, rows, el


def fft_form_rate(w, seconds: float, workers: int):
    """The method's CPU form (FP64, scipy FFT on `workers` threads; plan-time
    tables excluded) on consecutive 64-column blocks of the workload."""
    from oracle import fast
    plan = fast.FastPlan(_oracle_pointset(w), g=w.g if w.kind == "prime" else 0)
    A = w.A.astype(np.float64)
    block = min(64, w.t)
    cols = 0
    c0 = 0
    t0 = time.perf_counter()
    while True:
        c1 = min(w.t, c0 + block)
        plan.matmul(A[:, c0:c1], workers=workers)
        cols += c1 - c0
        c0 = c1 % w.t
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return plan.ps.out_rows * cols / el, cols, el


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return
    w = _make_workload(args.workload, 0, args.grid)
    for _ in range(args.warmup):
        oracle_rate(w, 0.5)
    vals = []
    rows_total = 0
    secs = []
    for _ in range(args.steps):
        v, rows, el = oracle_rate(w, args.ref_seconds)
        vals.append(v)
        rows_total += rows
        secs.append(el)
    value = float(statistics.median(vals))
    sample = (f"{rows_total} output rows x t={w.t} of {w.name} over {args.steps} steps "
              f"(~{args.ref_seconds:.0f} s each), FP64 numpy BLAS")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(secs)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "N": w.N, "s": w.s, "t": w.t, "map": w.map},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu_batch(args, rank, world, local_rank):
    """batch-64: 64 uneven problems in one qmc_batch_matmul (graph mode)."""
    import torch

    from paper_1501_06286_gb300 import build as qbuild
    from paper_1501_06286_gb300 import capi
    from paper_1501_06286_gb300.qmc import Batch, Plan

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    qbuild.build()
    lib = capi.load()
    ws = workloads.batch_64(seed=3)
    plans = [Plan.from_workload(w) for w in ws]
    As = [torch.from_numpy(w.A).to(dev) for w in ws]
    outs = [torch.empty((p.out_rows, w.t), dtype=torch.float32, device=dev) for p, w in zip(plans, ws)]
    batch = Batch(plans, [w.t for w in ws])
    batch.set_option("mode", args.batch_mode)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        batch.matmul(As, outs)
    barrier()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches0 = lib.qmc_kernel_launches()
    sampler = ClockSampler(local_rank)
    with sampler:
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            batch.matmul(As, outs)
            ends[k].record(stream)
        barrier()
    launches = lib.qmc_kernel_launches() - launches0
    assert batch.sync_status() == 0
    ms_local = float(np.mean([s.elapsed_time(e) for s, e in zip(starts, ends)]))
    t_local = torch.tensor([ms_local], device=dev, dtype=torch.float64)
    if world > 1:
        torch.distributed.all_reduce(t_local, op=torch.distributed.ReduceOp.MAX)
    ms = float(t_local.item())
    outputs = sum(p.out_rows * w.t for p, w in zip(plans, ws))
    value = world * outputs / (ms * 1e-3)
    # roofline of the batch as a whole: the three-pass design's bytes
    design = 0
    for p, w in zip(plans, ws):
        T = (w.t + 1) // 2
        work = 8 * p.L * T
        if p.info["L2"] == 1:
            design += 4 * w.s * w.t + 4 * p.out_rows * w.t
        else:
            design += 4 * w.s * w.t + 5 * work + 4 * p.out_rows * w.t
    peaks = _peaks()
    achieved = design / (ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": None,
                "kernel": f"batch ({args.batch_mode}): all passes of 64 problems",
                "algorithmic_bytes_per_launch": int(design), "peak_source": peaks["source"]}
    # end to end: copy every A in, run, copy every B out
    A_pin = [A.cpu().pin_memory() for A in As]
    B_pin = [torch.empty(o.shape, dtype=torch.float32).pin_memory() for o in outs]
    A_dev = [torch.empty_like(A) for A in As]

    def e2e_step():
        for a, ap in zip(A_dev, A_pin):
            a.copy_(ap, non_blocking=True)
        batch.matmul(A_dev, outs)
        for bp, o in zip(B_pin, outs):
            bp.copy_(o, non_blocking=True)

    e2e_step()
    barrier()
    t0 = time.perf_counter()
    n_e2e = 3
    for _ in range(n_e2e):
        e2e_step()
    barrier()
    e2e_s = (time.perf_counter() - t0) / n_e2e
    e2e = {"value": world * outputs / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(sum(4 * w.s * w.t for w in ws)),
           "d2h_bytes_per_step": int(4 * outputs), "ms_per_step": 1e3 * e2e_s}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, rows, el = oracle_rate(ws[0], args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
               "sample": f"{rows} output rows x t={ws[0].t} of batch problem 0 (N={ws[0].N}, s={ws[0].s}) "
                         f"in {el:.1f} s (FP64 numpy BLAS); rate per output"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "batch-64", "problems": len(ws), "outputs": int(outputs),
                           "mode": args.batch_mode,
                           "l2": "256 MB buffer written before every timed step (outside the events)",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": sampler.summary(), "dense_gemm": None}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_sweep_s(args):
    """FFT form vs dense-GEMM form over s at N = 65537, t = 512 (Φ^{-1}):
    one JSON line per s, both timed with CUDA events (median of 10)."""
    import torch

    from paper_1501_06286_gb300 import build as qbuild
    from paper_1501_06286_gb300.qmc import Plan

    torch.cuda.set_device(0)
    qbuild.build()
    torch.backends.cuda.matmul.allow_tf32 = False
    t = 512

    def timed(fn, reps=10):
        ts = []
        for _ in range(3):
            fn()
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    for s in (32, 64, 128, 256, 512, 1024, 2048, 4096):
        w = workloads.random_prime_case(65537, s, t, seed=s, map="phi_inv")
        plan = Plan.from_workload(w)
        A = torch.from_numpy(w.A).cuda()
        out = torch.empty((plan.out_rows, t), device="cuda")
        fft_ms = timed(lambda: plan.matmul(A, out=out))
        Y = plan.generate_points()
        Bd = torch.empty_like(out)
        dense_ms = timed(lambda: torch.matmul(Y, A, out=Bd))
        diff = ((out - Bd).abs().amax(dim=0) / out.abs().amax(dim=0).clamp_min(1e-30)).max().item()
        outputs = plan.out_rows * t
        print(json.dumps({"impl": "sweep", "workload": "random-65537", "N": 65537, "s": s, "t": t,
                          "fft_ms": fft_ms, "dense_ms": dense_ms, "fft_over_dense": dense_ms / fft_ms,
                          "fft_outputs_per_s": outputs / (fft_ms * 1e-3),
                          "dense_outputs_per_s": outputs / (dense_ms * 1e-3),
                          "max_colwise_rel_diff": diff}), flush=True)
        del Y, Bd, out, A, plan


def run_gpu(args, rank, world, local_rank):
    if args.sweep_s:
        return run_sweep_s(args)
    if args.workload == "batch-64":
        return run_gpu_batch(args, rank, world, local_rank)
    import ctypes as C

    import torch

    from paper_1501_06286_gb300 import build as qbuild
    from paper_1501_06286_gb300 import capi
    from paper_1501_06286_gb300.qmc import Plan

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    qbuild.build()
    lib = capi.load()

    w = _make_workload(args.workload, rank, args.grid)
    prec = "fp32_split" if args.split else "fp32"
    plan = Plan.from_workload(w, prec=prec)
    if args.kernel != "auto":
        plan.set_pass_kernel(args.kernel)
    A_host = w.A.astype(np.float64 if args.split else np.float32)
    A = torch.from_numpy(A_host).to(dev)
    out = torch.empty((plan.out_rows, w.t), dtype=torch.float32, device=dev)
    plan.reserve(w.t)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    # one step = the workload's whole hot path on device-resident inputs
    row_mean = w.epilogue == "row_mean"
    exp_loss = w.epilogue == "exp_loss"
    affine = w.epilogue in ("uniform", "lognormal")
    col_off = torch.from_numpy(w.extra["col_offset"]).to(dev) if affine else None
    apply_exp = bool(w.extra.get("apply_exp", False))
    dA = torch.empty((w.s, w.t), dtype=torch.float32, device=dev) if exp_loss else None

    def step():
        if affine:
            return plan.matmul_affine(A, col_off, apply_exp, out=out)
        if exp_loss:
            plan.matmul(A, out=out, exp_sum=True)
            return plan.matmul_backward(out, g_mode=1, dA=dA)
        if row_mean:
            return plan.matmul(A, out=out, row_mean=True)
        return plan.matmul(A, out=out)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()

    # ---- timed region: K steps, L2 flushed before each (outside the events)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    lib.qmc_plan_set_profiling(plan.handle, 1)
    lib.qmc_plan_read_profile(plan.handle, (C.c_double * capi.NUM_STAGES)(), (C.c_int32 * capi.NUM_STAGES)())
    launches0 = lib.qmc_kernel_launches()
    sampler = ClockSampler(local_rank)
    barrier()
    with sampler:
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            step()
            ends[k].record(stream)
        barrier()
    launches = lib.qmc_kernel_launches() - launches0
    stage_ms = (C.c_double * capi.NUM_STAGES)()
    stage_n = (C.c_int32 * capi.NUM_STAGES)()
    lib.qmc_plan_read_profile(plan.handle, stage_ms, stage_n)
    lib.qmc_plan_set_profiling(plan.handle, 0)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms_local = float(np.mean(step_ms))
    t_local = torch.tensor([ms_local], device=dev, dtype=torch.float64)
    if world > 1:
        torch.distributed.all_reduce(t_local, op=torch.distributed.ReduceOp.MAX)
    ms = float(t_local.item())
    outputs = plan.out_rows * w.t
    value = world * outputs / (ms * 1e-3)

    # ---- roofline of the dominant kernel (live events, same stream)
    stages = {capi.STAGES[i]: (stage_ms[i] / max(1, stage_n[i]), int(stage_n[i]))
              for i in range(capi.NUM_STAGES) if stage_n[i]}
    dom = max(stages, key=lambda k: stages[k][0] * stages[k][1])
    dom_ms, dom_n = stages[dom]
    T = (w.t + 1) // 2 if not args.split else w.t
    L = plan.L
    elem = 8  # complex64
    a_bytes = A_host.dtype.itemsize * w.s * w.t
    out_bytes = 4 * outputs
    work_bytes = elem * L * T
    g_bytes = 4 * outputs
    da_bytes = 4 * w.s * w.t
    dense_path = "dense_scatter" in stages  # P·A streamed first: pass A then reads the work array
    packed_bytes = 64 * w.s * ((T + 7) // 8)  # sparse first pass: A's rows by 8-column panel
    algo = {"fwd_scatter": (2 * work_bytes) if dense_path else (a_bytes + work_bytes),
            "sparse_pack": a_bytes + packed_bytes, "fwd_sparse": work_bytes,
            "dense_scatter": a_bytes + work_bytes, "fwd_spectral": 2 * work_bytes,
            "fwd_unpermute": work_bytes + out_bytes, "fwd_fused": a_bytes + out_bytes,
            "row0": a_bytes, "bwd_gather": g_bytes + work_bytes, "bwd_spectral": 2 * work_bytes,
            "bwd_scatter": work_bytes + da_bytes, "bwd_fused": g_bytes + da_bytes}
    peaks = _peaks()
    achieved = algo.get(dom, 0) / (dom_ms * 1e-3) / 1e9
    traffic = None
    tpath = os.path.join(ROOT, "profiles", f"traffic_{w.name}.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tr = json.load(f)
        # DRAM bytes per launch from one ncu capture, valid only for the
        # kernel sources the capture was taken from
        if tr.get("source_hash") == _source_hash(tr.get("sources")):
            traffic = tr.get("bytes_per_launch", {}).get(dom)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic,
                "kernel": dom, "kernel_ms": round(dom_ms, 4),
                "algorithmic_bytes_per_launch": int(algo.get(dom, 0)),
                "peak_source": peaks["source"],
                "stage_ms": {k: round(v[0], 4) for k, v in stages.items()}}

    # ---- end to end through the public API with host buffers
    A_pin = torch.from_numpy(A_host).pin_memory()
    B_pin = None if exp_loss else torch.empty((plan.out_rows, w.t), dtype=torch.float32).pin_memory()
    A_dev = torch.empty_like(A)
    e2e_steps = max(1, min(args.steps, 5))
    dA_pin = torch.empty((w.s, w.t), dtype=torch.float32).pin_memory() if exp_loss else None
    loss_pin = torch.empty(1, dtype=torch.float64).pin_memory()

    def e2e_step():
        # public API with host buffers: copy A in, run the step, copy the result out
        A_dev.copy_(A_pin, non_blocking=True)
        if exp_loss:
            _, _, es = plan.matmul(A_dev, out=out, exp_sum=True)
            g = plan.matmul_backward(out, g_mode=1, dA=dA)
            loss_pin.copy_(es, non_blocking=True)
            dA_pin.copy_(g, non_blocking=True)
            return
        if affine:
            plan.matmul_affine(A_dev, col_off, apply_exp, out=out)
        elif row_mean:
            plan.matmul(A_dev, out=out, row_mean=True)
        else:
            plan.matmul(A_dev, out=out)
        B_pin.copy_(out, non_blocking=True)

    for _ in range(2):
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    barrier()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    d2h = (8 + 4 * w.s * w.t) if exp_loss else int(B_pin.numel() * 4)
    e2e = {"value": world * outputs / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(A_pin.numel() * A_pin.element_size()),
           "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * e2e_s}

    # ---- same-GPU dense GEMM form (cuBLAS FP32, TF32 off) for the ratio
    # ---- the applications' whole step (Experiments 2 and 3): the product,
    # then the finite-element solves of every point and their mean, on
    # device-resident inputs; the paper's own time for the same N, M, s is
    # context only (Matlab on one Xeon)
    application = None
    if affine and rank == 0:
        from paper_1501_06286_gb300.qmc import fe_solve_mean
        fe_kind = "tridiag" if w.epilogue == "uniform" else "midpoint"
        M = (w.t + 3) // 2 if fe_kind == "tridiag" else w.t

        def app_step():
            plan.matmul_affine(A, col_off, apply_exp, out=out)
            return fe_solve_mean(out, M, fe_kind)

        for _ in range(2):
            app_step()
        napp = max(1, min(args.steps, 5))
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True)) for _ in range(napp)]
        barrier()
        for e0, e1, e2 in ev:
            flush.zero_()
            e0.record(stream)
            plan.matmul_affine(A, col_off, apply_exp, out=out)
            e1.record(stream)
            fe_solve_mean(out, M, fe_kind)
            e2.record(stream)
        barrier()
        app_ms = float(np.mean([e0.elapsed_time(e2) for e0, _, e2 in ev]))
        solve_ms = float(np.mean([e1.elapsed_time(e2) for _, e1, e2 in ev]))
        paper = {("uniform", 4001): 19.678, ("lognormal", 4001): 15.203}.get((w.epilogue, w.N))
        application = {"what": f"product + {w.N} tridiagonal FE solves (M={M}) + mean, FP64 solves",
                       "ms_per_step": app_ms, "solve_ms": solve_ms,
                       "paper_fast_s": paper if M == 2 * w.N and w.s == M else None,
                       "paper_hardware": "Matlab R2013b, one Xeon E5-2650v2 (context only)"}

    dense = None
    if not args.no_dense and rank == 0:
        torch.backends.cuda.matmul.allow_tf32 = False
        Y = plan.generate_points()
        Af = A.float()
        Bd = torch.matmul(Y, Af)
        dAd = torch.empty_like(Af) if exp_loss else None

        def dense_step():
            # the same work as step(): forward GEMM, and for the exp loss
            # the cotangent exp(B)/(rows t) and the adjoint GEMM Yᵀ G
            torch.matmul(Y, Af, out=Bd)
            if affine:
                Bd.add_(col_off)
                if apply_exp:
                    Bd.exp_()
            if exp_loss:
                G = torch.exp(Bd) / float(Bd.numel())
                torch.matmul(Y.t(), G, out=dAd)

        dense_step()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        reps = 2
        for _ in range(reps):
            dense_step()
        ev1.record()
        torch.cuda.synchronize()
        dms = ev0.elapsed_time(ev1) / reps
        step()
        torch.cuda.synchronize()
        scale = out.abs().amax(dim=0).clamp_min(1e-30)
        diff = (out - Bd).abs().amax(dim=0) / scale
        dense = {"value": outputs / (dms * 1e-3), "unit": UNIT, "ms_per_step": dms,
                 "kind": ("cuBLAS SGEMM (TF32 off) on Y materialised by qmc_generate_points"
                          + (", forward + exp + adjoint GEMM" if exp_loss else "")
                          + (", + column offsets" + (" + exp" if apply_exp else "") if affine else "")),
                 "fft_over_dense": (outputs / (ms * 1e-3)) / (outputs / (dms * 1e-3)),
                 "max_colwise_rel_diff_fft_vs_dense": float(diff.max().item())}
        del Y, Bd

    # ---- CPU oracle baseline (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, rows, el = oracle_rate(w, args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
               "sample": f"{rows} output rows x t={w.t} of {w.name} in {el:.1f} s (FP64 numpy BLAS)"}
        fv, fcols, fel = fft_form_rate(w, max(2.0, args.cpu_seconds / 4), cpu_cores())
        cpu["fft_form"] = {"value": fv, "unit": UNIT, "cores": cpu_cores(),
                           "kind": "the method's CPU form (oracle.fast: FP64 scipy FFT)",
                           "sample": f"all {plan.out_rows} output rows x {fcols} columns of {w.name} "
                                     f"in {fel:.1f} s, 64-column blocks"}

    clocks = sampler.summary()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": w.name, "N": w.N, "s": w.s, "t": w.t, "map": w.map,
                           "prec": prec, "L": plan.L, "L1": plan.info["L1"], "L2": plan.info["L2"],
                           "l2": "256 MB buffer written before every timed step (outside the events)",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clocks, "dense_gemm": dense}
        if application is not None:
            line["application"] = application
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _source_hash(files=None) -> str:
    """Hash of the kernel sources a traffic capture was taken from: the
    listed files (paths relative to the repository), or all of csrc/."""
    import hashlib
    h = hashlib.sha256()
    if files is None:
        csrc = os.path.join(ROOT, "paper_1501_06286_gb300", "csrc")
        files = [os.path.join("paper_1501_06286_gb300", "csrc", fn) for fn in sorted(os.listdir(csrc))]
    for fn in files:
        with open(os.path.join(ROOT, fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="gauss-65537")
    ap.add_argument("--grid", type=int, default=None,
                    help="node grid of field-786433 / f2-65536 (smaller cases for ncu captures)")
    ap.add_argument("--split", action="store_true", help="FP64 A as hi+lo FP32")
    ap.add_argument("--kernel", default="auto", choices=["auto", "generic", "register", "pipelined"])
    ap.add_argument("--batch-mode", default="graph", choices=["graph", "persistent"])
    ap.add_argument("--sweep-s", action="store_true",
                    help="FFT vs dense GEMM over s at N=65537, t=512 (one JSON line per s)")
    ap.add_argument("--no-dense", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=6.0)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
