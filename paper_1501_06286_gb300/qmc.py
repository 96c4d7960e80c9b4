"""Python binding of libqmcfft: plans, products, adjoint, batches.

Every step of the product runs in the library's CUDA kernels; this module
only marshals arguments (device pointers of torch tensors, the current CUDA
stream) and raises on a non-zero status.  There is no CPU fallback.
"""

from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import capi


def _stream_handle(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def _check_matrix(x: torch.Tensor, name: str) -> None:
    if not x.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if x.dim() != 2:
        raise ValueError(f"{name} must be 2-D")
    if x.stride(1) != 1:
        raise ValueError(f"{name} must be row-major (unit column stride)")


class Plan:
    """A fast-product plan: the point set, its tables and its spectrum.

    kind        'prime' (rank-1 lattice, prime N), 'f2' (polynomial lattice, N = 2^m),
                'fb' (polynomial lattice over F_b, N = b^m, b prime) or 'pset'
                (Korobov p-set of Section 2.2, N = K prime)
    gen         z_j (prime), q_j bit polynomials (f2), q_j base-b encodings (fb),
                or e_j with gen_is_exponent; None for a p-set, which takes `s` instead
    map         'identity' | 'centred' | 'phi_inv' | 'tent'
    row0        'auto' | 'include' | 'exclude'
    order       'conventional' | 'circulant'
    prec        'fp32' | 'fp32_split' (FP64 A split into hi + lo FP32)
    g, P        primitive root / modulus; 0 lets the library choose the smallest
    shift       diagonal shift Δ in [0, 1) of every coordinate (Remark 2)
    base        the prime b of an 'fb' plan
    """

    def __init__(self, kind: str, N: int, gen, map: str = "centred", row0: str = "auto",
                 order: str = "conventional", prec: str = "fp32", g: int = 0, P: int = 0,
                 gen_is_exponent: bool = False, shift: float = 0.0, s: int | None = None,
                 base: int = 0, stream=None):
        self._lib = capi.load()
        d = capi.QmcDesc()
        if kind == "pset":
            # Korobov p-set (Section 2.2): N = K prime, s coordinates, no generator
            if gen is not None or s is None:
                raise ValueError("a p-set plan takes s and no generator")
            self._gen = None
            d.s = int(s)
            d.gen_host = None
        else:
            gen = np.ascontiguousarray(np.asarray(gen, dtype=np.int64))
            self._gen = gen
            d.s = int(gen.shape[0])
            d.gen_host = gen.ctypes.data_as(C.POINTER(C.c_int64))
        d.kind = capi.KIND[kind]
        d.N = int(N)
        d.modulus_P = int(P)
        d.g = int(g)
        d.gen_is_exponent = int(bool(gen_is_exponent))
        d.map = capi.MAP[map]
        d.row0 = capi.ROW0[row0]
        d.order = capi.ORDER[order]
        d.prec = capi.PREC[prec]
        d.shift = float(shift)
        d.base = int(base)
        h = C.c_void_p()
        torch.cuda.init()
        capi.check(self._lib.qmc_plan_create(C.byref(h), C.byref(d), C.c_void_p(_stream_handle(stream))),
                   "qmc_plan_create")
        self._h = h
        self.kind, self.map, self.row0, self.order, self.prec = kind, map, row0, order, prec
        self.shift = float(shift)
        info = capi.QmcInfo()
        capi.check(self._lib.qmc_plan_info(self._h, C.byref(info)), "qmc_plan_info")
        self.info = {f: getattr(info, f) for f, _ in capi.QmcInfo._fields_}
        self.N = int(info.N)
        self.L = int(info.L)
        self.s = int(info.s)
        self.out_rows = int(info.out_rows)

    # ------------------------------------------------------------------
    @classmethod
    def from_workload(cls, w, prec: str = "fp32", order: str = "conventional", stream=None):
        return cls(w.kind, w.N, w.gen, map=w.map, row0=w.row0, order=order, prec=prec, g=w.g,
                   P=w.P, gen_is_exponent=w.gen_is_exponent, shift=getattr(w, "shift", 0.0),
                   base=w.extra.get("base", 0), stream=stream)

    @property
    def handle(self):
        return self._h

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.qmc_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------
    def exponents(self) -> np.ndarray:
        e = np.empty(self.s, dtype=np.int32)
        capi.check(self._lib.qmc_plan_exponents(self._h, e.ctypes.data_as(C.POINTER(C.c_int32))),
                   "qmc_plan_exponents")
        return e

    def table(self, name: str) -> np.ndarray:
        L, s = self.L, self.s
        shapes = {"pow": (np.int32, L), "log": (np.int32, self.N), "exponents": (np.int32, s),
                  "out_row": (np.int32, L), "zeta": (np.float64, L), "spectrum64": (np.float64, 2 * L),
                  "row_ptr": (np.int32, L + 1), "jlist": (np.int32, s)}
        dt, n = shapes[name]
        out = np.empty(n, dtype=dt)
        capi.check(self._lib.qmc_plan_copy_table(self._h, capi.TABLE[name], out.ctypes.data_as(C.c_void_p),
                                                 out.nbytes), "qmc_plan_copy_table")
        if name == "spectrum64":
            out = out[0::2] + 1j * out[1::2]
        return out

    def reserve(self, t_max: int) -> None:
        capi.check(self._lib.qmc_plan_reserve(self._h, int(t_max)), "qmc_plan_reserve")

    def set_pass_kernel(self, kind: str) -> None:
        """'auto' | 'generic' | 'register' (see qmc_plan_set_option)."""
        capi.check(self._lib.qmc_plan_set_option(self._h, capi.OPT_PASS_KERNEL, capi.KERNEL[kind]),
                   "qmc_plan_set_option")

    def set_row_mean_mode(self, mode: str) -> None:
        """'linear' (r = Y·(A·1/t)) or 'fused' (atomic row sums in the last pass)."""
        capi.check(self._lib.qmc_plan_set_option(self._h, capi.OPT_ROW_MEAN, capi.ROW_MEAN[mode]),
                   "qmc_plan_set_option")

    def set_first_pass(self, mode: str) -> None:
        """'auto' | 'transform' | 'sparse': how a two-pass forward product forms
        its first FFT pass (see qmc_first_pass in include/qmc.h)."""
        capi.check(self._lib.qmc_plan_set_option(self._h, capi.OPT_FIRST_PASS, capi.FIRST_PASS[mode]),
                   "qmc_plan_set_option")

    def set_fft_split(self, L1: int) -> None:
        """Re-factors the transform as L = L1·(L/L1) (0: the default split)
        and rebuilds the tables that depend on it (synchronous)."""
        capi.check(self._lib.qmc_plan_set_option(self._h, capi.OPT_FFT_SPLIT, int(L1)), "qmc_plan_set_option")
        info = capi.QmcInfo()
        capi.check(self._lib.qmc_plan_info(self._h, C.byref(info)), "qmc_plan_info")
        self.info = {f: getattr(info, f) for f, _ in capi.QmcInfo._fields_}

    def sync_status(self, stream=None) -> int:
        return self._lib.qmc_plan_sync_status(self._h, C.c_void_p(_stream_handle(stream)))

    # ------------------------------------------------------------------
    def matmul(self, A: torch.Tensor, out: torch.Tensor | None = None, row_mean: bool = False,
               exp_sum: bool = False, stream=None):
        """B = Y·A.  Returns out, or (out, row_mean, exp_sum) when requested."""
        _check_matrix(A, "A")
        if A.dtype not in (torch.float32, torch.float64):
            raise ValueError("A must be float32 or float64")
        t = A.shape[1]
        if A.shape[0] != self.s:
            raise ValueError(f"A must have s={self.s} rows")
        if out is None:
            out = torch.empty((self.out_rows, t), dtype=torch.float32, device=A.device)
        _check_matrix(out, "out")
        rm = torch.empty(self.out_rows, dtype=torch.float32, device=A.device) if row_mean else None
        es = torch.empty(1, dtype=torch.float64, device=A.device) if exp_sum else None
        rc = self._lib.qmc_matmul(self._h, _ptr(A), A.stride(0), t,
                                  capi.DTYPE_F64 if A.dtype == torch.float64 else capi.DTYPE_F32,
                                  _ptr(out), out.stride(0), _ptr(rm), _ptr(es),
                                  C.c_void_p(_stream_handle(stream)))
        capi.check(rc, "qmc_matmul")
        if row_mean or exp_sum:
            return out, rm, es
        return out

    def matmul_affine(self, A: torch.Tensor, col_offset: torch.Tensor | None = None, apply_exp: bool = False,
                      out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """B = exp?(col_offset + Y·A) (Sections 3.2 and 3.3)."""
        _check_matrix(A, "A")
        if A.dtype not in (torch.float32, torch.float64):
            raise ValueError("A must be float32 or float64")
        t = A.shape[1]
        if A.shape[0] != self.s:
            raise ValueError(f"A must have s={self.s} rows")
        if col_offset is not None and (col_offset.dtype != torch.float32 or col_offset.numel() != t
                                       or not col_offset.is_contiguous()):
            raise ValueError("col_offset must be a contiguous float32 vector of length t")
        if out is None:
            out = torch.empty((self.out_rows, t), dtype=torch.float32, device=A.device)
        _check_matrix(out, "out")
        rc = self._lib.qmc_matmul_affine(self._h, _ptr(A), A.stride(0), t,
                                         capi.DTYPE_F64 if A.dtype == torch.float64 else capi.DTYPE_F32,
                                         _ptr(col_offset), int(bool(apply_exp)), _ptr(out), out.stride(0),
                                         C.c_void_p(_stream_handle(stream)))
        capi.check(rc, "qmc_matmul_affine")
        return out

    def matmul_backward(self, G: torch.Tensor, g_mode: int = 0, dA: torch.Tensor | None = None,
                        stream=None) -> torch.Tensor:
        """dA = Yᵀ·G (g_mode 0), or Yᵀ·exp(G)/(rows·t) with G holding B (g_mode 1)."""
        _check_matrix(G, "G")
        if G.dtype != torch.float32 or G.shape[0] != self.out_rows:
            raise ValueError("G must be float32 with out_rows rows")
        t = G.shape[1]
        if dA is None:
            dA = torch.empty((self.s, t), dtype=torch.float32, device=G.device)
        _check_matrix(dA, "dA")
        rc = self._lib.qmc_matmul_backward(self._h, _ptr(G), G.stride(0), t, int(g_mode), _ptr(dA),
                                           dA.stride(0), C.c_void_p(_stream_handle(stream)))
        capi.check(rc, "qmc_matmul_backward")
        return dA

    def generate_points(self, stream=None) -> torch.Tensor:
        Y = torch.empty((self.out_rows, self.s), dtype=torch.float32, device="cuda")
        capi.check(self._lib.qmc_generate_points(self._h, _ptr(Y), Y.stride(0),
                                                 C.c_void_p(_stream_handle(stream))),
                   "qmc_generate_points")
        return Y


class Batch:
    """Many plans multiplied in one call (see qmc_batch_matmul)."""

    def __init__(self, plans: list[Plan], t: list[int], stream=None):
        self._lib = capi.load()
        self.plans = list(plans)
        self.t = [int(x) for x in t]
        arr = (C.c_void_p * len(plans))(*[p.handle.value for p in plans])
        tt = (C.c_int32 * len(plans))(*self.t)
        h = C.c_void_p()
        capi.check(self._lib.qmc_batch_create(C.byref(h), arr, tt, len(plans),
                                              C.c_void_p(_stream_handle(stream))), "qmc_batch_create")
        self._h = h

    def matmul(self, As: list[torch.Tensor], outs: list[torch.Tensor], stream=None) -> None:
        n = len(self.plans)
        for A, o in zip(As, outs):
            _check_matrix(A, "A")
            _check_matrix(o, "out")
        ap = (C.c_void_p * n)(*[A.data_ptr() for A in As])
        op = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
        la = (C.c_int64 * n)(*[A.stride(0) for A in As])
        lo = (C.c_int64 * n)(*[o.stride(0) for o in outs])
        capi.check(self._lib.qmc_batch_matmul(self._h, ap, la, op, lo, C.c_void_p(_stream_handle(stream))),
                   "qmc_batch_matmul")

    def set_option(self, name: str, value) -> None:
        """'mode' ('graph' | 'persistent'), 'branches', 'wait_limit_us', 'test_block_item'."""
        if name == "mode":
            value = capi.BATCH_MODE[value]
        capi.check(self._lib.qmc_batch_set_option(self._h, capi.BATCH_OPT[name], int(value)),
                   "qmc_batch_set_option")

    def sync_status(self, stream=None) -> int:
        return self._lib.qmc_batch_sync_status(self._h, C.c_void_p(_stream_handle(stream)))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.qmc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fe_solve_mean(B: torch.Tensor, M: int, kind: str = "tridiag", g_hat: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    """Finite-element step of Sections 3.2 / 3.3 (qmc_fe_solve_mean): for
    every row of B (one QMC point), solve the tridiagonal stiffness system of
    size M-1 and return the mean of the solutions (float64, M-1).  kind
    'tridiag': rows hold the diagonal then the super-diagonal (2M-3 floats,
    Experiment 2); 'midpoint': rows hold the coefficient at the M element
    midpoints (Experiment 3).  g_hat: float64 right-hand side (default ones)."""
    _check_matrix(B, "B")
    if B.dtype != torch.float32:
        raise ValueError("B must be float32")
    lib = capi.load()
    n_sys = B.shape[0]
    need = int(lib.qmc_fe_work_bytes(n_sys, int(M)))
    work = torch.empty(max(need, 8), dtype=torch.uint8, device=B.device)
    u = torch.empty(int(M) - 1, dtype=torch.float64, device=B.device)
    if g_hat is not None and (g_hat.dtype != torch.float64 or g_hat.numel() != M - 1 or not g_hat.is_contiguous()):
        raise ValueError("g_hat must be a contiguous float64 vector of length M-1")
    rc = lib.qmc_fe_solve_mean(_ptr(B), B.stride(0), n_sys, int(M), capi.FE_KIND[kind], _ptr(g_hat),
                               _ptr(work), work.numel(), _ptr(u), C.c_void_p(_stream_handle(stream)))
    capi.check(rc, "qmc_fe_solve_mean")
    return u
