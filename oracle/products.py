"""Dense FP64 products with the QMC matrix Y (oracle; test infrastructure).

Section 1: B = Y·A with Y the N x s matrix whose rows are the quadrature
points; the QMC estimate of the integral is (1/N) sum_n f(b_n).  The oracle
computes the product from its definition: rows of Y are materialised in
blocks (``PointSet.Y_rows``) and multiplied in float64 with numpy's matmul
(a library primitive used as one step).  Output rows follow the point set's
conventional order, with row 0 dropped when the row-0 policy excludes it.

Applications, each one written out from its definition:
  * Section 3.1, Eq. (5): z_n = y_n A + mu (here mu = 0);
  * Sections 3.2 / 3.3: b_n = y_n A is then reduced (the per-row mean over
    the field's t grid nodes is r_n = (1/t) sum_k B_nk);
  * loss l(A) = mean_{n,k} exp(B_nk), its gradient dl/dA = Y_outᵀ G with
    G = exp(B) / (rows * t).
"""

from __future__ import annotations

import numpy as np

from .points import PointSet

DEFAULT_BLOCK = 2048


def matmul_rows(ps: PointSet, A: np.ndarray, out_rows) -> np.ndarray:
    """B[out_rows, :] = Y[out_rows, :] · A, FP64."""
    A = np.asarray(A, dtype=np.float64)
    if A.ndim == 1:
        A = A[:, None]
    if A.shape[0] != ps.s:
        raise ValueError("A must have s rows")
    n = ps.output_row_to_n(out_rows)
    return ps.Y_rows(n) @ A


def matmul(ps: PointSet, A: np.ndarray, block: int = DEFAULT_BLOCK) -> np.ndarray:
    """B = Y·A over all output rows, FP64, Y materialised block by block."""
    A = np.asarray(A, dtype=np.float64)
    if A.ndim == 1:
        A = A[:, None]
    rows = ps.out_rows
    out = np.empty((rows, A.shape[1]), dtype=np.float64)
    for r0 in range(0, rows, block):
        r1 = min(rows, r0 + block)
        out[r0:r1] = matmul_rows(ps, A, np.arange(r0, r1))
    return out


def adjoint(ps: PointSet, G: np.ndarray, block: int = DEFAULT_BLOCK) -> np.ndarray:
    """Yᵀ·G (s x t), the gradient of <Y·A, G> with respect to A."""
    G = np.asarray(G, dtype=np.float64)
    if G.ndim == 1:
        G = G[:, None]
    rows = ps.out_rows
    if G.shape[0] != rows:
        raise ValueError("G must have out_rows rows")
    out = np.zeros((ps.s, G.shape[1]), dtype=np.float64)
    for r0 in range(0, rows, block):
        r1 = min(rows, r0 + block)
        Yb = ps.Y_rows(ps.output_row_to_n(np.arange(r0, r1)))
        out += Yb.T @ G[r0:r1]
    return out


def row_mean(B: np.ndarray) -> np.ndarray:
    """r_n = (1/t) sum_k B_nk."""
    return B.mean(axis=1)


def exp_mean_loss(B: np.ndarray) -> float:
    """l = mean over all entries of exp(B)."""
    return float(np.exp(B).mean())


def exp_mean_loss_grad_B(B: np.ndarray) -> np.ndarray:
    """dl/dB = exp(B) / (rows * t)."""
    return np.exp(B) / B.size


def exp_mean_loss_and_grad(ps: PointSet, A: np.ndarray):
    """Loss l(A) = mean exp(Y A) and dl/dA = Yᵀ exp(Y A)/(rows*t)."""
    B = matmul(ps, A)
    return exp_mean_loss(B), adjoint(ps, exp_mean_loss_grad_B(B))
