"""Korobov p-set of Section 2.2 (oracle; test infrastructure).

The union of all Korobov lattice point sets for a prime K (Hua and Wang):
    x_{n,g} = ({n g^0 / K}, {n g^1 / K}, ..., {n g^{s-1} / K}),  n, g = 1..K-1,
N = (K-1)^2 points; y_{n,g} = φ(x_{n,g}) with one map φ in every
coordinate.  Conventional output order: the point (n, g) is row
(g-1)(K-1) + (n-1), i.e. K-1 blocks of K-1 rows, block g holding the
Korobov lattice with generator (1, g, g^2, ...).

Section 2.2 reorders with a primitive element β: n -> β^{-(n-1)} and
g -> β^{(g-1)}.  Block g of the reordered matrix is then the lattice of
Section 2.1 with exponents c_{g,j} = (j-1)(g-1) + 1 (mod K-1), so
Y'_g = Z·P_g with the one circulant Z of the sequence z_k = φ({β^k/K}).
The formula for c_{g,j} places "mod (K-1)" ambiguously; since β has order
K-1 only c mod (K-1) matters for the points, and this module uses the
0-based exponent e_{g,j} = ((j-1)(g-1)) mod (K-1) in [0, K-2].
"""

from __future__ import annotations

import numpy as np

from . import numtheory
from .points import phi, shifted


class PSet:
    """Korobov p-set for prime K, s coordinates, map φ, diagonal shift Δ."""

    def __init__(self, K: int, s: int, map: str, shift: float = 0.0):
        if not numtheory.is_prime(K):
            raise ValueError("K must be prime")
        self.K, self.s, self.map, self.shift = int(K), int(s), map, float(shift)
        self.L = self.K - 1
        # φ({v/K + Δ}) for the K grid values v/K
        self._phi_table = np.array([phi(shifted(v / self.K, self.shift), map) for v in range(self.K)],
                                   dtype=np.float64)

    @property
    def out_rows(self) -> int:
        return self.L * self.L

    def numerators(self, rows) -> np.ndarray:
        """v with x = v/K for conventional rows (len(rows) x s): row
        (g-1)(K-1) + (n-1) is the point n·(1, g, g^2, ...) mod K."""
        rows = np.asarray(rows, dtype=np.int64)
        g = rows // self.L + 1
        n = rows % self.L + 1
        out = np.empty((len(rows), self.s), dtype=np.int64)
        gp = np.ones(len(rows), dtype=np.int64)       # g^j mod K
        for j in range(self.s):
            out[:, j] = (n * gp) % self.K
            gp = (gp * g) % self.K
        return out

    def Y_rows(self, rows) -> np.ndarray:
        return self._phi_table[self.numerators(rows)]

    def Y(self) -> np.ndarray:
        return self.Y_rows(np.arange(self.out_rows))


def matmul(ps: PSet, A: np.ndarray, block: int = 4096) -> np.ndarray:
    """B = Y·A over all (K-1)^2 rows, FP64, Y materialised block by block."""
    A = np.asarray(A, dtype=np.float64)
    if A.ndim == 1:
        A = A[:, None]
    out = np.empty((ps.out_rows, A.shape[1]), dtype=np.float64)
    for r0 in range(0, ps.out_rows, block):
        r1 = min(ps.out_rows, r0 + block)
        out[r0:r1] = ps.Y_rows(np.arange(r0, r1)) @ A
    return out


def exponents(K: int, s: int, g: int) -> list[int]:
    """e_{g,j} = ((j-1)(g-1)) mod (K-1), j = 1..s (0-based c_{g,j} - 1)."""
    return [((j - 1) * (g - 1)) % (K - 1) for j in range(1, s + 1)]


def reordered_block(K: int, s: int, beta: int, g: int) -> np.ndarray:
    """x_{n,g} of Section 2.2 for n = 1..K-1 (first displayed form):
    ({β^{-(n-1)} β^{(j-1)(g-1)} / K})_j.  Row index n-1."""
    binv = numtheory.inverse_mod(beta, K)
    out = np.empty((K - 1, s), dtype=np.float64)
    for n in range(1, K):
        a = pow(binv, n - 1, K)
        for j in range(1, s + 1):
            out[n - 1, j - 1] = (a * pow(beta, (j - 1) * (g - 1), K)) % K / K
    return out
