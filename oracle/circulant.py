"""The circulant factorisation Y' = Z·P written out (oracle; test infrastructure).

Section 2.1: with beta (``g``) primitive mod N,
    z_k = φ({beta^k / N}),  k in Z, period N-1,
    Z   = the (N-1)x(N-1) circulant whose first row is z_0..z_{N-2} and
          whose every next row is the previous one shifted right by one,
          i.e. Z[r][c] = z_{(c-r) mod (N-1)} (0-based),
    P   = (p_{k,j}), p_{k,j} = 1 iff k = c_j  (0-based: row e_j = c_j - 1),
and Eq. (3) states Y' = Z·P, Y' being rows 1..N-1 of Y in the reordered
order.  The product Z·a' is computed "using FFT"; the paper does not write
the FFT form out.  Since Z[r][c] = z_{c-r}, (Z a')_r = sum_c z_{c-r} a'_c is
a circular correlation, so with the DFT X_k = sum_n x_n e^{-2 pi i n k/L}:
    Z a' = IDFT( conj(DFT(z)) * DFT(a') )     (z real).
This module gives the explicit O(L^2) DFT so that tests can pin that
reading without any FFT library.
"""

from __future__ import annotations

import numpy as np

from . import f2, fb, points


def generator_sequence_prime(N: int, g: int, kind: str, delta: float = 0.0) -> np.ndarray:
    """z_k = φ({g^k/N + Δ}), k = 0..N-2 (Section 2.1; Δ the diagonal shift
    of Remark 2, 0 for the unshifted set)."""
    out = np.empty(N - 1, dtype=np.float64)
    v = 1
    for k in range(N - 1):
        out[k] = points.phi(points.shifted(v / N, delta), kind)
        v = (v * g) % N
    return out


def generator_sequence_f2(P: int, kind: str, delta: float = 0.0) -> np.ndarray:
    """z_k = φ({v_m(x^k mod P / P) + Δ}), k = 0..2^m-2 (Remark 1 with x
    primitive)."""
    m = f2.degree(P)
    L = (1 << m) - 1
    out = np.empty(L, dtype=np.float64)
    v = 1
    for k in range(L):
        out[k] = points.phi(points.shifted(f2.v_m(v, P), delta), kind)
        v = f2.mod(v << 1, P)
    return out


def generator_sequence_fb(P: list[int], b: int, kind: str, delta: float = 0.0) -> np.ndarray:
    """z_k = φ({v_m(x^k mod P / P) + Δ}), k = 0..b^m-2, over F_b (Remark 1
    with x primitive); P as coefficients, lowest first."""
    m = fb.degree(P)
    L = b ** m - 1
    out = np.empty(L, dtype=np.float64)
    v = [1]
    for k in range(L):
        out[k] = points.phi(points.shifted(fb.v_m_numerator(v, P, b) / b ** m, delta), kind)
        v = fb.divmod_poly([0] + v, P, b)[1]
    return out


def reordered_conventional_index_fb(P: list[int], b: int) -> list[int]:
    """Conventional index n of circulant row r over F_b: n(x) = x^{-r} mod P
    read as a base-b integer (r = 0..b^m-2)."""
    m = fb.degree(P)
    L = b ** m - 1
    return [fb.encode(fb.x_power((L - r) % L, P, b), b) for r in range(L)]


def circulant_Z(zeta: np.ndarray) -> np.ndarray:
    """Z[r][c] = zeta[(c - r) mod L] (the display of Z in Section 2.1)."""
    L = len(zeta)
    r = np.arange(L)[:, None]
    c = np.arange(L)[None, :]
    return zeta[(c - r) % L]


def selector_P(e, L: int) -> np.ndarray:
    """P[k][j] = 1 iff k = e_j (0-based form of p_{k,j} = 1 iff k = c_j)."""
    P = np.zeros((L, len(e)), dtype=np.float64)
    for j, ej in enumerate(e):
        P[int(ej), j] = 1.0
    return P


def scatter_add(e, A: np.ndarray, L: int) -> np.ndarray:
    """a' = P·A: row e_j of the result accumulates row j of A."""
    out = np.zeros((L,) + A.shape[1:], dtype=np.float64)
    for j, ej in enumerate(e):
        out[int(ej)] += A[j]
    return out


def collision_adds(e) -> int:
    """Number of additions P·a needs: s minus the number of distinct e_j."""
    return len(e) - len(set(int(v) for v in e))


def dft(x: np.ndarray) -> np.ndarray:
    """Explicit O(L^2) DFT along axis 0: X_k = sum_n x_n exp(-2 pi i n k / L).

    The phase index n*k is reduced mod L in exact integers before the
    float64 exponential so that large L does not lose the angle.
    """
    L = x.shape[0]
    n = np.arange(L)
    W = np.exp(-2j * np.pi * ((n[:, None] * n[None, :]) % L) / L)
    return W @ x


def idft(X: np.ndarray) -> np.ndarray:
    L = X.shape[0]
    n = np.arange(L)
    W = np.exp(2j * np.pi * ((n[:, None] * n[None, :]) % L) / L)
    return (W @ X) / L


def spectrum(zeta: np.ndarray) -> np.ndarray:
    """The multiplier of the correlation: conj(DFT(zeta)) / L (explicit DFT)."""
    return np.conj(dft(zeta)) / len(zeta)


def circulant_apply_dft(zeta: np.ndarray, a_prime: np.ndarray) -> np.ndarray:
    """Z·a' through the explicit DFT form (reading stated in the module doc)."""
    H = np.conj(dft(zeta))
    if a_prime.ndim == 2:
        H = H[:, None]
    return idft(H * dft(a_prime))


def spectrum_fft(zeta: np.ndarray) -> np.ndarray:
    """conj(DFT(zeta))/L with numpy's FFT as the DFT step (for L too large
    for the explicit O(L^2) form; numpy's FFT is pinned against ``dft``)."""
    return np.conj(np.fft.fft(zeta)) / len(zeta)

