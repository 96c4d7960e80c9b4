"""The fast product of Section 2.1 on the CPU, FP64 (oracle; test infrastructure).

This is the method itself written out step by step in float64, as a second,
independent route to B = Y·A beside the dense product of ``products``; the
tests check the two against each other, and the benchmark times this one as
the CPU form of the method.  It shares nothing with the GPU library.

Steps (Section 2.1, Eq. (3)), with L = N - 1 (F_2: L = 2^m - 1):
  1. e_j = log_g z_j (F_2: q_j = x^{e_j}); P·A is the scatter-add
     a'_u = Σ_{e_j = u} A_j  (one row of the L x t array per position u);
  2. Z·a' with Z[r][c] = ζ_{(c-r) mod L}, ζ_k = φ({g^k/N}) (F_2:
     φ(v_m(x^k mod P / P))), a circular correlation evaluated "using FFT":
         Z a' = IDFT( conj(DFT ζ) ⊙ DFT a' )
     (real input, so the real FFT of numpy/scipy is the DFT step);
  3. circulant row r is the point with conventional index g^{-r} mod N
     (F_2: n(x) = x^{-r} mod P read as an integer); rows go back to the
     conventional order;
  4. row 0, if kept, is φ(0)·Σ_j A_j.
With the diagonal shift of Remark 2 every coordinate x becomes {x + Δ}, so
ζ_k = φ({g^k/N + Δ}) and row 0 is φ(Δ)·Σ_j A_j.
"""

from __future__ import annotations

import numpy as np

from . import circulant, f2, numtheory
from .points import PointSet

try:  # scipy's FFT takes a worker count; numpy's is the fallback
    import scipy.fft as _fft

    def _rfft(x, workers):
        return _fft.rfft(x, axis=0, workers=workers)

    def _irfft(X, n, workers):
        return _fft.irfft(X, n=n, axis=0, workers=workers)
except ImportError:  # pragma: no cover
    def _rfft(x, workers):
        return np.fft.rfft(x, axis=0)

    def _irfft(X, n, workers):
        return np.fft.irfft(X, n=n, axis=0)


class FastPlan:
    """Plan-time part of the method: exponents, generator sequence ζ, its
    spectrum and the circulant-row -> output-row map."""

    def __init__(self, ps: PointSet, g: int = 0):
        self.ps = ps
        N = ps.N
        if ps.kind == "prime":
            self.g = g or numtheory.smallest_primitive_root(N)
            self.L = N - 1
            self.e = np.array(numtheory.exponents(ps.gen, self.g, N), dtype=np.int64)
            self.zeta = circulant.generator_sequence_prime(N, self.g, ps.map, ps.shift)
            ginv = numtheory.inverse_mod(self.g, N)
            n_of_r = np.empty(self.L, dtype=np.int64)
            v = 1
            for r in range(self.L):
                n_of_r[r] = v
                v = (v * ginv) % N
        else:
            P = ps.P
            self.g = 0
            self.L = N - 1
            lg = f2.log_table(P)
            self.e = np.array([lg[q] for q in ps.gen], dtype=np.int64)
            self.zeta = circulant.generator_sequence_f2(P, ps.map, ps.shift)
            # x^{-r} = x^{(L - r) mod L}
            pw = np.empty(self.L, dtype=np.int64)
            v = 1
            for k in range(self.L):
                pw[k] = v
                v = f2.mod(v << 1, P)
            n_of_r = pw[(self.L - np.arange(self.L)) % self.L]
        # conventional index n -> output row (row 0 dropped or kept)
        self.out_row = n_of_r if ps.has_row0 else n_of_r - 1
        # conj(DFT ζ) over the rfft half-spectrum
        self.spec = np.conj(np.fft.rfft(self.zeta))

    def matmul(self, A: np.ndarray, workers: int = 1) -> np.ndarray:
        """B = Y·A (out_rows x t) by steps 1-4 of the module docstring."""
        A = np.asarray(A, dtype=np.float64)
        if A.ndim == 1:
            A = A[:, None]
        ps = self.ps
        a_prime = np.zeros((self.L, A.shape[1]), dtype=np.float64)
        np.add.at(a_prime, self.e, A)
        Ba = _irfft(self.spec[:, None] * _rfft(a_prime, workers), self.L, workers)
        B = np.empty((ps.out_rows, A.shape[1]), dtype=np.float64)
        B[self.out_row] = Ba
        if ps.has_row0:
            B[0] = ps.phi0 * A.sum(axis=0)
        return B


def matmul_fft(ps: PointSet, A: np.ndarray, g: int = 0, workers: int = 1) -> np.ndarray:
    """One-shot form of ``FastPlan(ps, g).matmul(A, workers)``."""
    return FastPlan(ps, g).matmul(A, workers)
