"""Benchmark of the fast QMC product B = Y·A on GB300.

Default workload (field-786433, the largest single-GPU configuration): a
rank-1 lattice with N = 786433 (N - 1 = 3·2^18), s = 2048, t = 4225 (a 65 x 65
grid of nodes), centred map, A_jk = j^-2 sin(jπx_k1) sin(jπx_k2) (the
affine-parametric field of Section 3.2 / Section 4, Experiment 2), FP32
path, with the per-row mean of the field.  Other workloads: --workload
gauss-65537 (Φ^{-1} points, Cholesky factor of min(i,k)/s, Section 3.1 and
Experiment 1's shape), f2-65536 (polynomial lattice over F_2, exp loss and
its gradient), lattice-257, batch-64 and the finite-element workloads of
Experiments 2 and 3.

One step = one forward product (scatter-add, FFT, spectral product,
inverse FFT, un-permute, epilogue) over the whole batch of t columns.  Prints one JSON
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
# Dense comparator on tensor cores: cuBLAS FP32 GEMM with the BF16x9
# emulation (each FP32 operand split into three BF16 parts, products on the
# tensor cores, FP32 accumulation), called through ctypes on row-major
# torch tensors.  A library GEMM, used only for the dense form.
# ---------------------------------------------------------------------------
class CublasFp32Emulated:
    OP_N, OP_T = 0, 1
    R_32F = 0
    COMPUTE_32F_EMULATED_16BFX9 = 78
    EMULATION_EAGER = 2
    GEMM_DEFAULT = -1

    def __init__(self):
        import ctypes as C
        lib = None
        for name in ("libcublas.so.13", "/usr/local/cuda/lib64/libcublas.so.13", "libcublas.so"):
            try:
                lib = C.CDLL(name)
                break
            except OSError:
                continue
        if lib is None:
            raise RuntimeError("libcublas not found")
        self.C = C
        self.lib = lib
        self.handle = C.c_void_p()
        self._check(lib.cublasCreate_v2(C.byref(self.handle)), "cublasCreate")
        self._check(lib.cublasSetEmulationStrategy(self.handle, self.EMULATION_EAGER),
                    "cublasSetEmulationStrategy")
        lib.cublasGemmEx.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                     C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int,
                                     C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                     C.c_int]
        self.one = C.c_float(1.0)
        self.zero = C.c_float(0.0)

    @staticmethod
    def _check(rc, what):
        if rc != 0:
            raise RuntimeError(f"{what} failed: cuBLAS status {rc}")

    def _gemm(self, opa, opb, m, n, k, a, lda, b, ldb, c, ldc, stream):
        C = self.C
        self._check(self.lib.cublasSetStream_v2(self.handle, C.c_void_p(stream.cuda_stream)),
                    "cublasSetStream")
        self._check(self.lib.cublasGemmEx(self.handle, opa, opb, m, n, k, C.byref(self.one),
                                          C.c_void_p(a.data_ptr()), self.R_32F, lda,
                                          C.c_void_p(b.data_ptr()), self.R_32F, ldb, C.byref(self.zero),
                                          C.c_void_p(c.data_ptr()), self.R_32F, ldc,
                                          self.COMPUTE_32F_EMULATED_16BFX9, self.GEMM_DEFAULT),
                    "cublasGemmEx")

    def matmul(self, Y, A, out, stream):
        """out = Y·A, all row-major FP32 (out N x t, Y N x s, A s x t): the
        column-major product outᵀ = Aᵀ·Yᵀ."""
        N, s = Y.shape
        t = A.shape[1]
        self._gemm(self.OP_N, self.OP_N, t, N, s, A, A.stride(0), Y, Y.stride(0), out, out.stride(0),
                   stream)

    def matmul_tn(self, Y, G, out, stream):
        """out = Yᵀ·G (out s x t, Y N x s, G N x t), row-major: the
        column-major product outᵀ = Gᵀ·Y."""
        N, s = Y.shape
        t = G.shape[1]
        self._gemm(self.OP_N, self.OP_T, t, s, N, G, G.stride(0), Y, Y.stride(0), out, out.stride(0),
                   stream)


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


def _colwise(got, ref) -> float:
    """max over columns of max_n |got - ref| / max_n |ref| (a column whose
    reference is all zero must be exactly zero, else inf)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.ndim == 1:
        ref = ref[:, None]
        got = got.reshape(ref.shape)
    scale = np.abs(ref).max(axis=0)
    diff = np.abs(got - ref).max(axis=0)
    nz = scale > 0
    if np.any(diff[~nz] > 0):
        return float("inf")
    return float((diff[nz] / scale[nz]).max()) if np.any(nz) else 0.0


def oracle_errors(w, plan, A, A_host, out, dev, args):
    """Error of the GPU results against the FP64 oracle on this workload,
    measured once outside the timed region: the product on sampled output
    rows across all t columns (every row for lattice-257), the row mean, the
    split precision of the field workload, and for the exp-loss workload the
    loss and the whole gradient dA."""
    import torch

    from oracle import products
    from paper_1501_06286_gb300.qmc import Plan

    ps = _oracle_pointset(w)
    if plan.out_rows <= 4096:
        rows = np.arange(plan.out_rows)
    else:
        rng = np.random.default_rng(11)
        pick = rng.choice(plan.out_rows, 61, replace=False)
        rows = np.unique(np.concatenate([[0, 1, plan.out_rows - 1], pick]))
    rows_t = torch.from_numpy(rows).to(dev)
    A64 = A_host.astype(np.float64)
    ref_lin = products.matmul_rows(ps, A64, rows)
    res = {"measure": ("max over columns of max_n |B - B_oracle| / max_n |B_oracle|, FP64 oracle, "
                       f"{len(rows)} output rows x all {w.t} columns"),
           "rows": rows}
    prec = "fp32_split" if args.split else "fp32"
    if w.epilogue in ("uniform", "lognormal"):
        off = w.extra["col_offset"].astype(np.float64)
        apply_exp = bool(w.extra.get("apply_exp", False))
        ref = off[None, :] + ref_lin
        if apply_exp:
            ref = np.exp(ref)
        plan.matmul_affine(A, torch.from_numpy(w.extra["col_offset"]).to(dev), apply_exp, out=out)
        res[prec + ("_exp_affine" if apply_exp else "_affine")] = _colwise(out[rows_t].cpu().numpy(), ref)
        res["ref_rows"] = ref
        return res
    rm_ref = products.matmul_rows(ps, A64.mean(axis=1)[:, None], rows)[:, 0]
    _, rm, _ = plan.matmul(A, out=out, row_mean=True)
    res[prec] = _colwise(out[rows_t].cpu().numpy(), ref_lin)
    res["row_mean_" + prec] = _colwise(rm[rows_t].cpu().numpy(), rm_ref)
    res["ref_rows"] = ref_lin
    if w.name.startswith("field-786433") and not args.split:
        # the same field through the split hi+lo precision (FP64 A)
        grid = {"grid": args.grid} if args.grid else {}
        w64 = workloads.field_786433(seed=2, dtype=np.float64, **grid)
        p64 = Plan.from_workload(w64, prec="fp32_split")
        A64_dev = torch.from_numpy(w64.A).to(dev)
        _, rm64, _ = p64.matmul(A64_dev, out=out, row_mean=True)
        res["fp32_split"] = _colwise(out[rows_t].cpu().numpy(), products.matmul_rows(ps, w64.A, rows))
        res["row_mean_fp32_split"] = _colwise(
            rm64[rows_t].cpu().numpy(),
            products.matmul_rows(ps, w64.A.mean(axis=1)[:, None], rows)[:, 0])
        p64.close()
        del A64_dev, rm64
        torch.cuda.empty_cache()
    if w.epilogue == "exp_loss":
        ref_B = products.matmul(ps, A64)
        ref_loss = products.exp_mean_loss(ref_B)
        ref_grad = products.adjoint(ps, products.exp_mean_loss_grad_B(ref_B))
        _, _, es = plan.matmul(A, out=out, exp_sum=True)
        dA = plan.matmul_backward(out, g_mode=1)
        loss = es.item() / (plan.out_rows * w.t)
        res["forward_all_rows"] = _colwise(out.cpu().numpy(), ref_B)
        res["loss_rel"] = abs(loss - ref_loss) / abs(ref_loss)
        res["gradient"] = _colwise(dA.cpu().numpy(), ref_grad)
        res["ref_grad"] = ref_grad
    return res


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
    """batch-64: 64 uneven problems in one qmc_batch_matmul (graph or persistent mode)."""
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
    # roofline of the batch as a whole: algorithmic bytes (read every A,
    # write every B), and the three-pass design's bytes (work arrays
    # included) as the bandwidth the batch sustains
    design = 0
    algo = 0
    for p, w in zip(plans, ws):
        T = (w.t + 1) // 2
        work = 8 * p.L * T
        algo += 4 * w.s * w.t + 4 * p.out_rows * w.t
        if p.info["L2"] == 1:
            design += 4 * w.s * w.t + 4 * p.out_rows * w.t
        else:
            design += 4 * w.s * w.t + 5 * work + 4 * p.out_rows * w.t
    peaks = _peaks()
    achieved = algo / (ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": None,
                "kernel": f"batch ({args.batch_mode}): all passes of 64 problems",
                "algorithmic_bytes_per_launch": int(algo), "peak_source": peaks["source"],
                "algorithmic_frac": round(achieved / peaks["hbm_gbs"], 4),
                "design_bytes_per_launch": int(design),
                "achieved_bandwidth_frac": round(design / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4)}
    # error against the FP64 oracle: every problem, sampled rows, all columns
    errors = None
    if rank == 0 and not args.no_oracle_error:
        from oracle import products
        worst = 0.0
        for b, (p, w, o) in enumerate(zip(plans, ws, outs)):
            ps = _oracle_pointset(w)
            rng = np.random.default_rng(100 + b)
            rows = np.unique(np.concatenate([[0, p.out_rows - 1],
                                             rng.choice(p.out_rows, min(p.out_rows, 30), replace=False)]))
            ref = products.matmul_rows(ps, w.A.astype(np.float64), rows)
            worst = max(worst, _colwise(o[torch.from_numpy(rows).to(dev)].cpu().numpy(), ref))
        errors = {"measure": ("max over the 64 problems and their columns of max_n |B - B_oracle| / "
                              "max_n |B_oracle|, FP64 oracle, 32 sampled rows per problem x all columns"),
                  "fp32": worst}
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
                "clocks": sampler.summary(), "dense_gemm": None, "error_vs_oracle": errors}
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
    try:
        emu = CublasFp32Emulated()
    except Exception:
        emu = None

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
        stream = torch.cuda.current_stream()
        emu_ms = timed(lambda: emu.matmul(Y, A, Bd, stream)) if emu is not None else None
        diff_emu = ((out - Bd).abs().amax(dim=0) / out.abs().amax(dim=0).clamp_min(1e-30)).max().item()
        outputs = plan.out_rows * t
        print(json.dumps({"impl": "sweep", "workload": "random-65537", "N": 65537, "s": s, "t": t,
                          "fft_ms": fft_ms, "dense_ms": dense_ms, "fft_over_dense": dense_ms / fft_ms,
                          "dense_bf16x9_ms": emu_ms,
                          "fft_over_dense_bf16x9": (emu_ms / fft_ms) if emu_ms else None,
                          "fft_outputs_per_s": outputs / (fft_ms * 1e-3),
                          "dense_outputs_per_s": outputs / (dense_ms * 1e-3),
                          "max_colwise_rel_diff": diff,
                          "max_colwise_rel_diff_bf16x9": diff_emu if emu_ms else None}), flush=True)
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
    # pinned host buffers of the end-to-end steps, allocated first (two
    # result buffers used alternately, see below)
    e2e_shape = (w.s, w.t) if w.epilogue == "exp_loss" else (plan.out_rows, w.t)
    res_pin = [torch.empty(e2e_shape, dtype=torch.float32, pin_memory=True) for _ in range(2)]
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

    # ---- one step captured in a CUDA graph (the steady state the metric is
    # quoted in); the library's launches during the capture are the graph's
    # kernels.  Eager launches if the capture is not possible.
    graph, graph_launches, launch_mode = None, 0, "eager"
    if not args.no_graph:
        try:
            side = torch.cuda.Stream()
            side.wait_stream(stream)
            with torch.cuda.stream(side):
                step()
            stream.wait_stream(side)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            l0 = lib.qmc_kernel_launches()
            with torch.cuda.graph(g):
                step()
            graph_launches = lib.qmc_kernel_launches() - l0
            torch.cuda.synchronize()
            for _ in range(args.warmup):
                g.replay()
            graph, launch_mode = g, "CUDA graph replay"
        except Exception as e:  # noqa: BLE001 - any capture failure: time eager launches
            launch_mode = f"eager (graph capture failed: {str(e)[:120]})"
        barrier()

    # ---- timed region: K steps, L2 flushed before each (outside the events)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches0 = lib.qmc_kernel_launches()
    sampler = ClockSampler(local_rank)
    barrier()
    with sampler:
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            if graph is not None:
                graph.replay()
            else:
                step()
            ends[k].record(stream)
        barrier()
    launches = graph_launches * args.steps if graph is not None else lib.qmc_kernel_launches() - launches0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]

    # ---- per-stage kernel times (the library's events on the launching
    # stream) over eager steps of the same work, L2 flushed likewise
    lib.qmc_plan_set_profiling(plan.handle, 1)
    lib.qmc_plan_read_profile(plan.handle, (C.c_double * capi.NUM_STAGES)(), (C.c_int32 * capi.NUM_STAGES)())
    for k in range(max(1, min(args.steps, 10))):
        flush.zero_()
        step()
    barrier()
    stage_ms = (C.c_double * capi.NUM_STAGES)()
    stage_n = (C.c_int32 * capi.NUM_STAGES)()
    lib.qmc_plan_read_profile(plan.handle, stage_ms, stage_n)
    lib.qmc_plan_set_profiling(plan.handle, 0)
    ms_local = float(np.mean(step_ms))
    t_local = torch.tensor([ms_local], device=dev, dtype=torch.float64)
    if world > 1:
        torch.distributed.all_reduce(t_local, op=torch.distributed.ReduceOp.MAX)
    ms = float(t_local.item())
    outputs = plan.out_rows * w.t
    value = world * outputs / (ms * 1e-3)

    # ---- roofline of the dominant kernel (live events, same stream)
    # Algorithmic bytes: the method's minimum traffic, read A and write B
    # (forward; plus the row means), read G and write dA (adjoint).  Each
    # forward pass kernel processes every output of the product in one
    # launch, so its per-launch algorithmic bytes are the product's; the
    # adjoint's passes likewise process all of G.  Design bytes: what the
    # kernel must move in this design (the L x T work array between passes),
    # which is what ncu's DRAM counters see.
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
    rm_bytes = 4 * plan.out_rows if row_mean else 0
    fwd_algo = a_bytes + out_bytes + rm_bytes
    bwd_algo = g_bytes + da_bytes
    step_algo = fwd_algo + (bwd_algo if exp_loss else 0)
    dense_path = "dense_scatter" in stages  # P·A streamed first: pass A then reads the work array
    packed_bytes = 64 * w.s * ((T + 7) // 8)  # sparse first pass: A's rows by 8-column panel
    design = {"fwd_scatter": (2 * work_bytes) if dense_path else (a_bytes + work_bytes),
              "sparse_pack": a_bytes + packed_bytes, "fwd_sparse": work_bytes,
              "dense_scatter": a_bytes + work_bytes, "fwd_spectral": 2 * work_bytes,
              "fwd_unpermute": work_bytes + out_bytes, "fwd_fused": a_bytes + out_bytes,
              "row0": a_bytes, "row_mean": a_bytes, "bwd_gather": g_bytes + work_bytes,
              "bwd_spectral": 2 * work_bytes, "bwd_scatter": work_bytes + da_bytes,
              "bwd_fused": g_bytes + da_bytes}
    algo_launch = bwd_algo if dom.startswith("bwd_") else (a_bytes if dom in ("row0", "row_mean") else fwd_algo)
    peaks = _peaks()
    achieved = algo_launch / (dom_ms * 1e-3) / 1e9
    achieved_design = design.get(dom, 0) / (dom_ms * 1e-3) / 1e9
    traffic = None
    tpath = os.path.join(ROOT, "profiles", f"traffic_{w.name}.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tr = json.load(f)
        # DRAM bytes per launch from one ncu capture, valid only for the
        # kernel sources the capture was taken from
        if tr.get("source_hash") == _source_hash(tr.get("sources")):
            traffic = tr.get("bytes_per_launch", {}).get(dom)
    step_achieved = step_algo / (ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic,
                "kernel": dom, "kernel_ms": round(dom_ms, 4),
                "algorithmic_bytes_per_launch": int(algo_launch),
                "algorithmic_bytes_per_output": round(algo_launch / outputs, 4),
                "peak_source": peaks["source"],
                "algorithmic_frac": round(step_achieved / peaks["hbm_gbs"], 4),
                "algorithmic_frac_what": "whole step: algorithmic bytes / ms_per_step / peak",
                "design_bytes_per_launch": int(design.get(dom, 0)),
                "achieved_bandwidth_frac": round(achieved_design / peaks["hbm_gbs"], 4),
                "achieved_bandwidth_what": ("dominant kernel: design bytes (work array included) / "
                                            "kernel time / peak, the DRAM bandwidth it sustains"),
                "stage_ms": {k: round(v[0], 4) for k, v in stages.items()}}

    # ---- end to end through the public API with host buffers: every step
    # copies its A in from pinned host memory, runs the step and copies its
    # result out to pinned host memory.  Consecutive steps overlap on two
    # streams (step k's device->host copy of B runs while step k+1 computes;
    # the host link, about 193 GB/s here, is the bound), each step with its
    # own device result and host buffer (two of each, used alternately)
    A_pin = torch.empty(A_host.shape, dtype=A.dtype, pin_memory=True)
    A_pin.copy_(torch.from_numpy(A_host))
    A_devs = [torch.empty_like(A) for _ in range(2)]
    if exp_loss:
        res_dev = [dA, torch.empty_like(dA)]
    else:
        res_dev = [out, torch.empty_like(out)]
    e2e_steps = max(1, min(args.steps, 8))
    loss_pin = torch.empty(1, dtype=torch.float64, pin_memory=True)
    rm_pin = torch.empty(plan.out_rows, dtype=torch.float32, pin_memory=True) if row_mean else None
    copy_stream = torch.cuda.Stream()
    copy_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(e2e_steps)]
    computed = [torch.cuda.Event() for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]

    def e2e_step(k):
        b = k % 2
        stream.wait_event(copied[b])           # this buffer's previous copy-out is over
        A_devs[b].copy_(A_pin, non_blocking=True)
        if exp_loss:
            _, _, es = plan.matmul(A_devs[b], out=out, exp_sum=True)
            plan.matmul_backward(out, g_mode=1, dA=res_dev[b])
            loss_pin.copy_(es, non_blocking=True)
        elif affine:
            plan.matmul_affine(A_devs[b], col_off, apply_exp, out=res_dev[b])
        elif row_mean:
            _, rm_dev, _ = plan.matmul(A_devs[b], out=res_dev[b], row_mean=True)
            rm_pin.copy_(rm_dev, non_blocking=True)
        else:
            plan.matmul(A_devs[b], out=res_dev[b])
        computed[b].record(stream)
        copy_stream.wait_event(computed[b])
        with torch.cuda.stream(copy_stream):
            copy_ev[k % len(copy_ev)][0].record(copy_stream)
            res_pin[b].copy_(res_dev[b], non_blocking=True)
            copy_ev[k % len(copy_ev)][1].record(copy_stream)
            copied[b].record(copy_stream)

    for k in range(2):
        e2e_step(k)
    barrier()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        e2e_step(k)
    barrier()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    copy_ms = float(np.mean([a.elapsed_time(b) for a, b in copy_ev]))
    d2h = (8 + 4 * w.s * w.t) if exp_loss else int(res_pin[0].numel() * 4) + (4 * plan.out_rows if row_mean else 0)
    e2e = {"value": world * outputs / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(A_pin.numel() * A_pin.element_size()),
           "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * e2e_s,
           "overlap": "two streams: step k's copy-out runs during step k+1's copy-in and compute",
           "copy_out_ms": copy_ms,
           "copy_out_gbs": res_pin[0].numel() * 4 / (copy_ms * 1e-3) / 1e9}

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
        how = ("defect correction (flux-form preconditioner, FP32 then FP32-pair steps), "
               "partitioned FP64 elimination for systems that do not settle" if fe_kind == "tridiag"
               else "flux form: row and column sums in FP32 pairs, combination and prefix sum in FP64")
        application = {"what": f"product + {w.N} tridiagonal FE solves (M={M}) + mean, {how}",
                       "ms_per_step": app_ms, "solve_ms": solve_ms,
                       "paper_fast_s": paper if M == 2 * w.N and w.s == M else None,
                       "paper_hardware": "Matlab R2013b, one Xeon E5-2650v2 (context only)"}

    # ---- error against the FP64 oracle (outside the timed region)
    errors = None
    if rank == 0 and not args.no_oracle_error:
        errors = oracle_errors(w, plan, A, A_host, out, dev, args)

    # ---- same-GPU dense GEMM forms on Y materialised by qmc_generate_points:
    # cuBLAS SGEMM (TF32 off, SIMT FP32) and cuBLAS FP32 with the BF16x9
    # emulation on the tensor cores; each timed and checked against the oracle
    dense = None
    if not args.no_dense and rank == 0:
        torch.backends.cuda.matmul.allow_tf32 = False
        Y = plan.generate_points()
        Af = A.float()
        Bd = torch.empty((plan.out_rows, w.t), dtype=torch.float32, device=dev)
        dAd = torch.empty_like(Af) if exp_loss else None
        try:
            emu = CublasFp32Emulated()
        except Exception as exc:  # library missing: report the SIMT form only
            emu = None
            emu_error = str(exc)

        # cuBLAS uses the BF16x9 emulation only on aligned operands: the
        # emulated form multiplies Y and A padded with zeros to multiples of 8
        # columns (Y) and rows and columns (A) into a B of the padded width
        # (the extra products are zeros)
        t_pad = -(-w.t // 8) * 8
        s_pad = -(-w.s // 8) * 8
        if s_pad != w.s:
            Y_pad = torch.zeros((plan.out_rows, s_pad), dtype=torch.float32, device=dev)
            Y_pad[:, :w.s] = Y
        else:
            Y_pad = Y
        if t_pad != w.t or s_pad != w.s:
            Af_pad = torch.zeros((s_pad, t_pad), dtype=torch.float32, device=dev)
            Af_pad[:w.s, :w.t] = Af
        else:
            Af_pad = Af
        Bd_pad = torch.empty((plan.out_rows, t_pad), dtype=torch.float32, device=dev) if t_pad != w.t else Bd

        def dense_step(form):
            # the same work as step(): forward GEMM, and for the exp loss
            # the cotangent exp(B)/(rows t) and the adjoint GEMM Yᵀ G
            if form == "sgemm":
                torch.matmul(Y, Af, out=Bd)
            else:
                emu.matmul(Y_pad, Af_pad, Bd_pad, stream)
                if Bd_pad is not Bd:
                    Bd.copy_(Bd_pad[:, :w.t])
            if affine:
                Bd.add_(col_off)
                if apply_exp:
                    Bd.exp_()
            if exp_loss:
                G = torch.exp(Bd) / float(Bd.numel())
                if form == "sgemm":
                    torch.matmul(Y.t(), G, out=dAd)
                else:
                    if t_pad != w.t or s_pad != w.s:
                        G_pad = torch.zeros((plan.out_rows, t_pad), dtype=torch.float32, device=dev)
                        G_pad[:, :w.t] = G
                        dA_pad = torch.empty((s_pad, t_pad), dtype=torch.float32, device=dev)
                        emu.matmul_tn(Y_pad, G_pad, dA_pad, stream)
                        dAd.copy_(dA_pad[:w.s, :w.t])
                    else:
                        emu.matmul_tn(Y, G, dAd, stream)

        forms = {}
        for form in ("sgemm", "bf16x9"):
            if form == "bf16x9" and emu is None:
                forms[form] = {"unavailable": emu_error}
                continue
            dense_step(form)
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 2
            ev0.record(stream)
            for _ in range(reps):
                dense_step(form)
            ev1.record(stream)
            torch.cuda.synchronize()
            dms = ev0.elapsed_time(ev1) / reps
            entry = {"value": outputs / (dms * 1e-3), "unit": UNIT, "ms_per_step": dms,
                     "kind": ("cuBLAS SGEMM (TF32 off, FP32 SIMT)" if form == "sgemm" else
                              "cuBLAS FP32 GEMM, BF16x9 emulation on the tensor cores "
                              "(CUBLAS_COMPUTE_32F_EMULATED_16BFX9; Y and A zero-padded to multiples of 8)")
                             + " on Y materialised by qmc_generate_points"
                             + (", forward + exp + adjoint GEMM" if exp_loss else "")
                             + (", + column offsets" + (" + exp" if apply_exp else "") if affine else ""),
                     "fft_over_dense": dms / ms}
            if errors is not None and "rows" in errors:
                rows_t = torch.from_numpy(errors["rows"]).to(dev)
                entry["error_vs_oracle"] = _colwise(Bd[rows_t].cpu().numpy(), errors["ref_rows"])
                if exp_loss and "ref_grad" in errors:
                    entry["gradient_error_vs_oracle"] = _colwise(dAd.cpu().numpy(), errors["ref_grad"])
            forms[form] = entry
        dense = {"forms": forms, "flops_per_step": 2.0 * plan.out_rows * w.s * w.t * (2 if exp_loss else 1)}
        del Y, Bd, Bd_pad, Af_pad, Y_pad
    if errors is not None:
        errors.pop("rows", None)
        errors.pop("ref_rows", None)
        errors.pop("ref_grad", None)

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
                           "launch": launch_mode,
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clocks, "dense_gemm": dense,
                "error_vs_oracle": errors}
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
    ap.add_argument("--workload", default="field-786433")
    ap.add_argument("--grid", type=int, default=None,
                    help="node grid of field-786433 / f2-65536 (smaller cases for ncu captures)")
    ap.add_argument("--split", action="store_true", help="FP64 A as hi+lo FP32")
    ap.add_argument("--kernel", default="auto", choices=["auto", "generic", "register", "pipelined"])
    ap.add_argument("--batch-mode", default="graph", choices=["graph", "persistent"])
    ap.add_argument("--sweep-s", action="store_true",
                    help="FFT vs dense GEMM over s at N=65537, t=512 (one JSON line per s)")
    ap.add_argument("--no-dense", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="time eager launches instead of CUDA graph replays")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-oracle-error", action="store_true",
                    help="skip the error against the FP64 oracle (measured outside the timed region)")
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
