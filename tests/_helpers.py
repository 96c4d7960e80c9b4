"""Shared helpers for the parity tests (error metrics and oracle set-up)."""

from __future__ import annotations

import numpy as np

from oracle import f2, fb, numtheory, points

TOL = 1e-5  # max relative error per column (∞-norm), FP32 path vs FP64 oracle


def colwise_rel_err(got: np.ndarray, ref: np.ndarray) -> float:
    """max over columns of max_n |got - ref| / max_n |ref|; a column whose
    reference is identically zero must come out exactly zero."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.ndim == 1:
        ref = ref[:, None]
        got = got.reshape(ref.shape)
    scale = np.abs(ref).max(axis=0)
    diff = np.abs(got - ref).max(axis=0)
    zero = scale == 0
    if np.any(zero):
        assert np.all(diff[zero] == 0), "non-zero output where the reference is zero"
    if np.all(zero):
        return 0.0
    return float((diff[~zero] / scale[~zero]).max())


def oracle_pointset(w, row0=None, map=None):
    """PointSet for a workload, built only from oracle arithmetic."""
    row0 = row0 or w.row0
    map = map or w.map
    if w.kind == "prime":
        return points.PointSet("prime", w.N, w.gen, map, row0, shift=w.shift)
    if w.kind == "fb":
        b, m = w.extra["base"], w.extra["m"]
        P = w.P or fb.encode(fb.smallest_primitive(m, b), b)
        return points.PointSet("fb", w.N, list(w.gen), map, row0, P=P, shift=w.shift, base=b)
    m = w.extra.get("m", int(np.log2(w.N)))
    P = f2.smallest_primitive(m) if not w.P else w.P
    gen = [f2.x_power_fast(int(e), P) for e in w.gen] if w.gen_is_exponent else list(w.gen)
    return points.PointSet("f2", w.N, gen, map, row0, P=P, shift=w.shift)


def conventional_output_rows(N, g, has_row0):
    """Output row of circulant row r under conventional order (prime)."""
    conv = points.reordered_conventional_index_prime(N, g)
    return np.array(conv) - (0 if has_row0 else 1)


def internal_order(L1: int, L2: int) -> np.ndarray:
    """Index map of the library's two-factor transform, which leaves the
    spectrum in digit-transposed order: slot k1*L2 + k2 holds DFT index
    k1 + L1*k2 (for L2 = 1 the order is natural)."""
    k1 = np.arange(L1)[:, None]
    k2 = np.arange(L2)[None, :]
    return (k1 + L1 * k2).reshape(-1)


class ColwiseErr:
    """colwise_rel_err accumulated over row blocks, for products too large to
    hold twice in host memory: per column the largest |got - ref| and the
    largest |ref| seen so far."""

    def __init__(self, ncols: int):
        self.diff = np.zeros(ncols)
        self.scale = np.zeros(ncols)

    def add(self, got: np.ndarray, ref: np.ndarray) -> None:
        got = np.asarray(got, dtype=np.float64)
        ref = np.asarray(ref, dtype=np.float64)
        np.maximum(self.diff, np.abs(got - ref).max(axis=0), out=self.diff)
        np.maximum(self.scale, np.abs(ref).max(axis=0), out=self.scale)

    def value(self) -> float:
        zero = self.scale == 0
        if np.any(zero):
            assert np.all(self.diff[zero] == 0), "non-zero output where the reference is zero"
        if np.all(zero):
            return 0.0
        return float((self.diff[~zero] / self.scale[~zero]).max())


def panel_columns(t: int, split: bool, middle: int | None = None) -> np.ndarray:
    """Real columns of A (and B) that cover whole 8-complex-column panels of
    the work array: the first two panels, one in the middle and the last two
    (the last one ragged when the panel count does not divide).  FP32 pairs
    real columns 2c, 2c+1 into complex column c (16 real columns a panel);
    the split precision carries one real column per complex column (8 a
    panel)."""
    per = 8 if split else 16
    panels = -(-t // per)
    mid = panels // 2 if middle is None else middle
    keep = sorted({0, 1, mid, panels - 2, panels - 1} & set(range(panels)))
    cols = []
    for p in keep:
        cols.extend(range(p * per, min(t, (p + 1) * per)))
    return np.array(cols, dtype=np.int64)


def oracle_row_blocks(ps, rhs: np.ndarray, block: int = 4096):
    """Yields (r0, r1, Y[r0:r1] · rhs) over every output row of the point
    set, FP64, from the oracle's definition of Y (rows materialised block by
    block)."""
    from oracle import products
    rhs = np.asarray(rhs, dtype=np.float64)
    for r0 in range(0, ps.out_rows, block):
        r1 = min(ps.out_rows, r0 + block)
        yield r0, r1, products.matmul_rows(ps, rhs, np.arange(r0, r1))
