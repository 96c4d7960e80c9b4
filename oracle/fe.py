"""Finite-element step of the paper's applications (oracle; test
infrastructure only).

Sections 3.2 and 3.3 and Experiments 2 and 3: after the product, each
quadrature point y_n gives a symmetric tridiagonal stiffness matrix B(y_n)
of size M-1 (hat functions φ_k at x_k = k/M on (0, 1), zero boundary
values); the linear system B(y_n) û^(n) = ĝ with ĝ = (1, ..., 1) is solved
for every n, and the estimate of the expected finite-element coefficients is
their mean ū = (1/N) Σ_n û^(n).

Two ways of reading B(y_n) from a row b of the product:
  * 'tridiag' (Experiment 2): b holds the M-1 diagonal entries b_{k,k},
    k = 1..M-1, then the M-2 off-diagonal entries b_{k,k+1}, k = 1..M-2
    (the columns a_0 + Y·a_{k,l} of Section 3.2);
  * 'midpoint' (Experiment 3): b holds the coefficient a(x_i, y_n) at the M
    element midpoints x_i = (i - 1/2)/M (the exp of Section 3.3's Θ), and
    the stiffness matrix is assembled with that one-point, equal-weight
    rule per element: element i = [x_{i-1}, x_i] adds M·a_i to b_{i-1,i-1}
    and b_{i,i} and -M·a_i to b_{i-1,i}, so b_{k,k} = M (a_k + a_{k+1}) and
    b_{k,k+1} = -M a_{k+1}.

The tridiagonal solve is Gaussian elimination without pivoting written out
for three bands (the Thomas algorithm), vectorised over the systems, in
float64.
"""

from __future__ import annotations

import numpy as np


def stiffness(b: np.ndarray, M: int, kind: str) -> tuple[np.ndarray, np.ndarray]:
    """(diag, off) of the stiffness matrices of the rows of b: diag is
    rows x (M-1), off is rows x (M-2) with off[:, k-1] = b_{k,k+1}."""
    b = np.atleast_2d(np.asarray(b, dtype=np.float64))
    if kind == "tridiag":
        if b.shape[1] < 2 * M - 3:
            raise ValueError("tridiag rows need 2M-3 entries")
        return b[:, : M - 1], b[:, M - 1: 2 * M - 3]
    if kind == "midpoint":
        if b.shape[1] < M:
            raise ValueError("midpoint rows need M entries")
        a = b[:, :M]
        diag = M * (a[:, : M - 1] + a[:, 1:M])      # elements k and k+1 of node k
        off = -M * a[:, 1: M - 1]                     # element k+1 joins nodes k, k+1
        return diag, off
    raise ValueError(kind)


def solve_tridiag(diag: np.ndarray, off: np.ndarray, rhs: np.ndarray) -> np.ndarray:
    """Solves the symmetric tridiagonal systems (rows of diag / off) for the
    right-hand side rhs (length M-1): forward elimination, back substitution."""
    diag = np.atleast_2d(np.asarray(diag, dtype=np.float64))
    off = np.atleast_2d(np.asarray(off, dtype=np.float64))
    rhs = np.asarray(rhs, dtype=np.float64)
    rows, n = diag.shape
    c = np.empty((rows, n))       # modified super-diagonal
    d = np.empty((rows, n))       # modified right-hand side
    c[:, 0] = (off[:, 0] / diag[:, 0]) if n > 1 else 0.0
    d[:, 0] = rhs[0] / diag[:, 0]
    for k in range(1, n):
        den = diag[:, k] - off[:, k - 1] * c[:, k - 1]
        c[:, k] = off[:, k] / den if k < n - 1 else 0.0
        d[:, k] = (rhs[k] - off[:, k - 1] * d[:, k - 1]) / den
    u = np.empty((rows, n))
    u[:, n - 1] = d[:, n - 1]
    for k in range(n - 2, -1, -1):
        u[:, k] = d[:, k] - c[:, k] * u[:, k + 1]
    return u


def mean_solution(B: np.ndarray, M: int, kind: str, rhs: np.ndarray | None = None) -> np.ndarray:
    """ū = (1/N) Σ_n û^(n) over the rows of B (Section 3.2's estimate of the
    expected finite-element coefficients), ĝ = 1 unless rhs is given."""
    diag, off = stiffness(B, M, kind)
    g = np.ones(M - 1) if rhs is None else np.asarray(rhs, dtype=np.float64)
    return solve_tridiag(diag, off, g).mean(axis=0)


def constant_coefficient_solution(M: int, a: float) -> np.ndarray:
    """Nodal values for a ≡ const and ĝ = 1: ĝ_k = ∫ g φ_k = 1 means g = M,
    the exact solution of -(a u')' = M, u(0) = u(1) = 0 is
    u = M x (1 - x) / (2a), and piecewise-linear elements reproduce it at
    the nodes in one dimension."""
    x = np.arange(1, M) / M
    return M * x * (1.0 - x) / (2.0 * a)
