"""Point sets, coordinate maps and the matrix Y (oracle; test infrastructure).

Section 2.1: a rank-1 lattice point set with prime N and generating vector
(z_1..z_s) in (Z_N^*)^s has points ({n z_1/N}, ..., {n z_s/N}),
n = 0..N-1 ("conventional order").  The quadrature points are
y_n = φ(x_n) with one univariate map φ applied to every coordinate; the
paper names φ = Φ^{-1} (inverse normal CDF), the tent map 1-|2x-1| and the
identity, and Section 4 (Experiment 2) uses the centred map x - 1/2.

Row 0 is the point x_0 = 0, so y_0 = (φ(0), ..., φ(0)) and
y_0·a = φ(0)·Σ_j a_j (Section 2.1).  For φ = Φ^{-1}, φ(0) = -inf; the
reading adopted here drops that row ("row-0 policy auto": keep row 0 iff
φ(0) is finite).

Remark 1: polynomial lattice rules over F_2 (see ``oracle.f2``) have points
x_{n,j} = v_m(n(x) q_j(x) / P(x)), n = 0..2^m-1; over F_b for a prime b
(kind 'fb', see ``oracle.fb``) the same with base-b digits, n = 0..b^m-1.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from statistics import NormalDist

import numpy as np

from . import f2, fb, numtheory

MAPS = ("identity", "centred", "tent", "phi_inv")

_ND = NormalDist()


def phi(x: float, kind: str) -> float:
    """The coordinate map φ of Section 2.1 (and the centred map of Section 4)."""
    if kind == "identity":
        return x
    if kind == "centred":
        return x - 0.5
    if kind == "tent":
        return 1.0 - abs(2.0 * x - 1.0)
    if kind == "phi_inv":
        if x <= 0.0:
            return -math.inf
        # statistics.NormalDist.inv_cdf: Wichura's AS241 algorithm in
        # float64, independent of the CUDA math library.
        return _ND.inv_cdf(x)
    raise ValueError(f"unknown map {kind!r}")


def shifted(x: float, delta: float) -> float:
    """{x + Δ} for x, Δ in [0, 1): one float64 addition and, when the sum
    reaches 1, one subtraction (the diagonal shift of Remark 2: the same Δ
    in every coordinate)."""
    y = x + delta
    return y - 1.0 if y >= 1.0 else y


def include_row0(kind: str, policy: str, delta: float = 0.0) -> bool:
    """Row-0 policy: 'include', 'exclude', or 'auto' (include iff φ at the
    row-0 point, {0 + Δ} = Δ, is finite)."""
    if policy == "include":
        return True
    if policy == "exclude":
        return False
    if policy == "auto":
        return math.isfinite(phi(delta, kind))
    raise ValueError(policy)


@dataclass
class PointSet:
    """A lattice (kind='prime') or polynomial lattice (kind='f2') point set.

    prime: N prime, gen = (z_1..z_s) with z_j in Z_N^*.
    f2:    N = 2^m, P primitive of degree m, gen = (q_1..q_s) as bit
           polynomials, 0 < q_j, deg q_j < m.
    fb:    N = b^m for a prime base b, P the integer encoding sum_i p_i b^i of
           a monic primitive polynomial of degree m over F_b, gen = (q_1..q_s)
           encoded the same way, 0 < q_j < b^m.
    """

    kind: str
    N: int
    gen: list
    map: str
    row0: str = "auto"
    P: int = 0
    shift: float = 0.0   # diagonal shift Δ in [0, 1): x -> {x + Δ} in every coordinate
    base: int = 2        # fb only: the prime b of F_b
    _phi_table: np.ndarray = field(default=None, repr=False)

    def __post_init__(self):
        self.gen = [int(v) for v in self.gen]
        if self.kind == "prime":
            if not numtheory.is_prime(self.N):
                raise ValueError("N must be prime")
            if any(v % self.N == 0 for v in self.gen):
                raise ValueError("z_j must lie in Z_N^*")
        elif self.kind == "f2":
            m = f2.degree(self.P)
            if self.N != (1 << m):
                raise ValueError("N must be 2^deg(P)")
            if any(v == 0 or f2.degree(v) >= m for v in self.gen):
                raise ValueError("q_j must be nonzero with degree < m")
        elif self.kind == "fb":
            b = self.base
            if not numtheory.is_prime(b):
                raise ValueError("the base must be prime")
            m = 0
            while b ** (m + 1) <= self.P:
                m += 1
            self._Pc = fb.decode(self.P, b, m + 1)
            if self._Pc[-1] != 1 or self.N != b ** m:
                raise ValueError("P must be monic of degree m with N = b^m")
            self._m = m
            if any(v <= 0 or v >= self.N for v in self.gen):
                raise ValueError("q_j must be nonzero with degree < m")
        else:
            raise ValueError(self.kind)
        # φ is only ever evaluated at the N grid values v/N, v = 0..N-1
        # (prime: {n z/N} = ((n z) mod N)/N; F_2: v_m(h/P) = k/2^m).  One
        # table of φ(v/N) is the map applied pointwise, computed once.
        # With a diagonal shift the table holds φ({v/N + Δ}).
        self.shift = float(self.shift)
        if not (0.0 <= self.shift < 1.0):
            raise ValueError("shift must lie in [0, 1)")
        self._phi_table = np.array([phi(shifted(v / self.N, self.shift), self.map)
                                    for v in range(self.N)], dtype=np.float64)

    @property
    def s(self) -> int:
        return len(self.gen)

    @property
    def has_row0(self) -> bool:
        return include_row0(self.map, self.row0, self.shift)

    @property
    def phi0(self) -> float:
        """φ at the row-0 point {0 + Δ} = Δ."""
        return phi(self.shift, self.map)

    @property
    def out_rows(self) -> int:
        return self.N if self.has_row0 else self.N - 1

    def point_numerators(self, n_rows) -> np.ndarray:
        """Integer numerators v with x_{n,j} = v/N for the given conventional
        indices n (shape len(n_rows) x s)."""
        n_rows = np.asarray(n_rows, dtype=np.int64)
        if self.kind == "prime":
            z = np.asarray(self.gen, dtype=np.int64)
            return (n_rows[:, None] * z[None, :]) % self.N
        if self.kind == "fb":
            return self._numerators_fb(n_rows)
        # F_2: h = n(x) q_j(x) mod P, then the m Laurent digits of h/P by
        # long division, vectorised over the rows.  The product mod P uses
        # distributivity: h = XOR over the set bits i of n of (x^i q_j mod P).
        m = f2.degree(self.P)
        P = self.P
        out = np.empty((len(n_rows), self.s), dtype=np.int64)
        bits = [((n_rows >> i) & 1).astype(bool) for i in range(m)]
        for j, q in enumerate(self.gen):
            h = np.zeros(len(n_rows), dtype=np.int64)
            for i in range(m):
                b_i = f2.mulmod(1 << i, q, P)
                h = np.where(bits[i], h ^ b_i, h)
            r = h.copy()
            num = np.zeros(len(n_rows), dtype=np.int64)
            for _ in range(m):
                r = r << 1
                u = (r >> m) & 1
                r = np.where(u == 1, r ^ P, r)
                num = (num << 1) | u
            out[:, j] = num
        return out

    def _numerators_fb(self, n_rows: np.ndarray) -> np.ndarray:
        """F_b: h = n(x) q_j(x) mod P by linearity over the base-b digits of
        n (h = sum_i n_i (x^i q_j mod P), coefficientwise mod b), then the
        Laurent digits of h/P by the long-division recurrence of
        ``fb.laurent_digits``, vectorised over the rows."""
        b, m, Pc = self.base, self._m, self._Pc
        digits = np.stack([(n_rows // b ** i) % b for i in range(m)], axis=1)  # rows x m
        out = np.empty((len(n_rows), self.s), dtype=np.int64)
        for j, q in enumerate(self.gen):
            qc = fb.decode(q, b, m)
            basis = np.zeros((m, m), dtype=np.int64)  # row i: coefficients of x^i q_j mod P
            for i in range(m):
                r = fb.mulmod(fb.decode(b ** i, b, m), qc, Pc, b)
                basis[i, :len(r)] = r
            h = (digits @ basis) % b                    # rows x m: coefficients h_0..h_{m-1}
            u = np.zeros((len(n_rows), m + 1), dtype=np.int64)
            num = np.zeros(len(n_rows), dtype=np.int64)
            for r in range(1, m + 1):
                acc = h[:, m - r].copy()
                for k in range(1, r):
                    acc -= Pc[m - r + k] * u[:, k]
                u[:, r] = acc % b
                num = num * b + u[:, r]
            out[:, j] = num
        return out

    def points(self, n_rows) -> np.ndarray:
        """x_n for conventional indices n (float64, exact multiples of 1/N),
        before the shift."""
        return self.point_numerators(n_rows).astype(np.float64) / self.N

    def Y_rows(self, n_rows) -> np.ndarray:
        """Rows y_n = φ(x_n) for conventional indices n."""
        return self._phi_table[self.point_numerators(n_rows)]

    def output_row_to_n(self, out_rows) -> np.ndarray:
        """Conventional point index n of each output row (conventional order)."""
        out_rows = np.asarray(out_rows, dtype=np.int64)
        return out_rows if self.has_row0 else out_rows + 1

    def Y(self) -> np.ndarray:
        """The full output-row matrix (out_rows x s).  Small cases only."""
        return self.Y_rows(self.output_row_to_n(np.arange(self.out_rows)))


def reordered_points_prime(N: int, g: int, e) -> np.ndarray:
    """The reordered points of Section 2.1: x_n = ({g^{e_j - (n-1)}/N})_j for
    n = 1..N-1 (e_j = c_j - 1).  Returned with row index n-1."""
    L = N - 1
    e = [int(v) for v in e]
    out = np.empty((L, len(e)), dtype=np.float64)
    for r in range(L):
        for j, ej in enumerate(e):
            out[r, j] = pow(g, (ej - r) % L, N) / N
    return out


def reordered_conventional_index_prime(N: int, g: int) -> list[int]:
    """Conventional index of reordered point n (n = 1..N-1): g^{-(n-1)} mod N
    (Section 2.1: the conventional index n is replaced by beta^{-(n-1)})."""
    ginv = numtheory.inverse_mod(g, N)
    return [pow(ginv, r, N) for r in range(N - 1)]
