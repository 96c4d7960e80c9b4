"""Seeded synthetic inputs for the fast QMC product (shared by tests and bench).

This module holds only the random draws and the input matrices of the five
workloads; it performs none of the method's arithmetic (no discrete logs,
no point construction, no transforms).  Each workload is described by its
sizes, the seeded draws that define its generating vector, and the matrix A.

The paper's experiments use synthetic inputs only (Section 4: a random
upper-triangular Cholesky factor; sine-expansion coefficients of an ODE
coefficient).  The shapes here follow those workloads:

  lattice-257        N=257, g=3, s=200, t=1, centred map, FP64 a_j = U(-1,1) j^-2
  gauss-65537        N=65537, s=t=4096, Korobov z_j = alpha^(j-1), Φ^{-1},
                     A = upper Cholesky factor of min(i,k)/s (Section 3.1)
  field-786433       N=786433, s=2048, t=4225 nodes of a 65x65 grid,
                     A_jk = j^-2 sin(j pi x1) sin(j pi x2), centred (Section 3.2)
  batch-64           64 uneven problems, N from six primes, centred map
  f2-65536           polynomial lattice over F_2 with N=2^16, s=1024, t=1089
                     nodes of a 33x33 grid, A_jk = j^-2 cos(j pi x1) cos(j pi x2),
                     Φ^{-1}, loss = mean exp(Y A) (Section 3.3 shape)

Seeds: numpy.random.default_rng(k) with k = 0..4 in the order above.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Primitive roots quoted with each prime workload (the smallest primitive
# element of Z_N^*; the test-suite checks each one independently).
PRIMITIVE_ROOT = {3: 2, 5: 2, 7: 3, 4001: 3, 16001: 3, 25601: 3, 17: 3, 257: 3, 7681: 17, 12289: 11, 40961: 3,
                  65537: 3, 786433: 10}

BATCH_PRIMES = (257, 7681, 12289, 40961, 65537, 786433)


@dataclass
class Workload:
    """One problem instance.

    kind        'prime' (rank-1 lattice, N prime) or 'f2' (polynomial lattice)
    N           number of points
    g           primitive root used for the generator (prime); 0 for f2
    P           modulus polynomial (f2; 0 = the library's smallest primitive)
    gen         z_j (prime) or e_j (when gen_is_exponent)
    exponents   the seeded e_j draws (None when the config draws z_j directly)
    A           s x t matrix (float32 or float64)
    shift       diagonal shift Δ in [0, 1) of every coordinate (Remark 2)
    """

    name: str
    kind: str
    N: int
    g: int
    P: int
    gen: np.ndarray
    gen_is_exponent: bool
    map: str
    row0: str
    A: np.ndarray
    epilogue: str = "none"
    exponents: np.ndarray | None = None
    extra: dict = field(default_factory=dict)
    shift: float = 0.0   # diagonal shift Δ of every coordinate (Remark 2)

    @property
    def s(self) -> int:
        return self.A.shape[0]

    @property
    def t(self) -> int:
        return self.A.shape[1]


def _sin_pi_frac(p: np.ndarray, d: int) -> np.ndarray:
    """sin(pi * p / d) for integer p, with exact integer range reduction so
    that multiples of d give exactly 0."""
    p = np.mod(p, 2 * d)
    sign = np.where(p >= d, -1.0, 1.0)
    p = np.mod(p, d)
    p = np.minimum(p, d - p)
    return sign * np.sin(np.pi * p / d)


def lattice_257(seed: int = 0, s: int = 200, N: int = 257, g: int | None = None) -> Workload:
    rng = np.random.default_rng(seed)
    g = PRIMITIVE_ROOT[N] if g is None else g
    e = rng.integers(0, N - 1, size=s)
    z = np.array([pow(g, int(v), N) for v in e], dtype=np.int64)
    j = np.arange(1, s + 1, dtype=np.float64)
    a = rng.uniform(-1.0, 1.0, size=s) * j ** -2.0
    return Workload("lattice-257", "prime", N, g, 0, z, False, "centred", "auto",
                    a[:, None].astype(np.float64), exponents=e)


def gauss_65537(seed: int = 1, s: int = 4096, t: int | None = None,
                N: int = 65537) -> Workload:
    """Section 3.1 with the Brownian covariance Sigma_ik = min(i,k)/s.

    The upper Cholesky factor of Sigma is exactly triu(ones)/sqrt(s), because
    min(i,k) = sum_{l <= min(i,k)} 1.  A Korobov vector z_j = alpha^(j-1) mod
    N with alpha = g^d, d odd, drawn from the seed.  With t < s the first t
    columns of the factor are used.
    """
    rng = np.random.default_rng(seed)
    g = PRIMITIVE_ROOT[N]
    L = N - 1
    d = 2 * int(rng.integers(0, L // 2)) + 1
    alpha = pow(g, d, N)
    z = np.array([pow(alpha, j, N) for j in range(s)], dtype=np.int64)
    e = np.array([(j * d) % L for j in range(s)], dtype=np.int64)
    t = s if t is None else t
    A = np.triu(np.ones((s, s), dtype=np.float64))[:, :t] / math.sqrt(s)
    return Workload("gauss-65537", "prime", N, g, 0, z, False, "phi_inv", "auto",
                    A.astype(np.float32), exponents=e, extra={"d": d, "alpha": alpha})


def field_786433(seed: int = 2, s: int = 2048, grid: int = 65, N: int = 786433,
                 dtype=np.float32) -> Workload:
    """Section 3.2 shape: A_jk = j^-2 sin(j pi x_k1) sin(j pi x_k2) on the
    grid x = i/(grid-1), node k = i1*grid + i2."""
    rng = np.random.default_rng(seed)
    g = PRIMITIVE_ROOT[N]
    L = N - 1
    e = rng.integers(0, L, size=s)
    z = np.array([pow(g, int(v), N) for v in e], dtype=np.int64)
    h = grid - 1
    i = np.arange(grid)
    j = np.arange(1, s + 1)
    S = _sin_pi_frac(np.outer(j, i), h)                # s x grid: sin(j pi i/h)
    A = (S[:, :, None] * S[:, None, :]).reshape(s, grid * grid)
    A = A * (j.astype(np.float64) ** -2.0)[:, None]
    return Workload("field-786433", "prime", N, g, 0, z, False, "centred", "auto",
                    A.astype(dtype), epilogue="row_mean", exponents=e)


def batch_64(seed: int = 3, count: int = 64, primes=BATCH_PRIMES,
             s_max: int = 4096, t_max: int = 512) -> list[Workload]:
    """64 uneven problems: N uniform over six primes,
    s = floor(exp(U(ln 64, ln s_max))), t = floor(exp(U(0, ln t_max))),
    e_j ~ U{0..N-2}, A ~ N(0,1) * j^-1.5 (float32), centred map."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        N = int(rng.choice(primes))
        s = int(math.floor(math.exp(rng.uniform(math.log(64), math.log(s_max)))))
        t = int(math.floor(math.exp(rng.uniform(0.0, math.log(t_max)))))
        g = PRIMITIVE_ROOT[N]
        e = rng.integers(0, N - 1, size=s)
        z = np.array([pow(g, int(v), N) for v in e], dtype=np.int64)
        j = np.arange(1, s + 1, dtype=np.float64)
        A = rng.standard_normal((s, t)) * (j ** -1.5)[:, None]
        out.append(Workload(f"batch-64[{b}]", "prime", N, g, 0, z, False, "centred",
                            "auto", A.astype(np.float32), exponents=e))
    return out


def f2_65536(seed: int = 4, m: int = 16, s: int = 1024, grid: int = 33) -> Workload:
    """Polynomial lattice over F_2 with N = 2^m: q_j = x^{e_j} mod P with the
    seeded e_j (passed as exponents), A_jk = j^-2 cos(j pi x_k1) cos(j pi x_k2)
    on x = i/(grid-1), Φ^{-1} map, loss = mean exp(Y A)."""
    rng = np.random.default_rng(seed)
    L = (1 << m) - 1
    e = rng.integers(0, L, size=s).astype(np.int64)
    h = grid - 1
    i = np.arange(grid)
    j = np.arange(1, s + 1)
    C = _sin_pi_frac(h // 2 - np.outer(j, i), h)       # cos(pi j i/h)
    A = (C[:, :, None] * C[:, None, :]).reshape(s, grid * grid)
    A = A * (j.astype(np.float64) ** -2.0)[:, None]
    return Workload("f2-65536", "f2", 1 << m, 0, 0, e, True, "phi_inv", "auto",
                    A.astype(np.float32), epilogue="exp_loss", exponents=e,
                    extra={"m": m})


def fb_case(b: int, m: int, s: int, t: int, seed: int, map: str = "centred",
            row0: str = "auto", dtype=np.float32) -> Workload:
    """Polynomial lattice over F_b (b prime), N = b^m: generating polynomials
    q_j drawn uniformly from the nonzero encodings 1..N-1 (collisions
    allowed), A ~ N(0,1) * j^-1 (modulus: the smallest primitive one)."""
    rng = np.random.default_rng(seed)
    N = b ** m
    q = rng.integers(1, N, size=s).astype(np.int64)
    j = np.arange(1, s + 1, dtype=np.float64)
    A = rng.standard_normal((s, t)) * (j ** -1.0)[:, None]
    return Workload(f"fb{b}-{N}-{s}x{t}", "fb", N, 0, 0, q, False, map, row0, A.astype(dtype),
                    extra={"m": m, "base": b})


def random_prime_case(N: int, s: int, t: int, seed: int, map: str = "centred",
                      row0: str = "auto", dtype=np.float32) -> Workload:
    """Small seeded case for parity tests: e_j ~ U{0..N-2} (collisions
    allowed), A ~ N(0,1)."""
    rng = np.random.default_rng(seed)
    g = PRIMITIVE_ROOT[N]
    e = rng.integers(0, N - 1, size=s)
    z = np.array([pow(g, int(v), N) for v in e], dtype=np.int64)
    A = rng.standard_normal((s, t))
    return Workload(f"random-{N}-{s}x{t}", "prime", N, g, 0, z, False, map, row0,
                    A.astype(dtype), exponents=e)


# ---------------------------------------------------------------------------
# The paper's applications (Sections 3.2, 3.3; Experiments 2 and 3): inputs of
# the affine product B = exp?(c + Y·A).
# ---------------------------------------------------------------------------
def fe_uniform_coefficients(M: int, s: int) -> tuple[np.ndarray, np.ndarray]:
    """Experiment 2 (uniform case): a(x, y) = 2 + Σ_j y_j j^{-3/2} sin(2πjx)
    on (0, 1), hat functions φ_k at x_k = k/M, k = 1..M-1.  Returns A (s x C)
    with the closed-form a_{j,k,l} of the experiment for j = 1..s and the
    column offsets a_{0,k,l} (C = 2M-3 columns: the diagonal k = 1..M-1,
    then the super-diagonal (k, k+1), k = 1..M-2; the stiffness matrix is
    symmetric and tridiagonal)."""
    j = np.arange(1, s + 1, dtype=np.float64)[:, None]
    k = np.arange(1, M, dtype=np.int64)[None, :]
    amp = M * M / (np.pi * j ** 2.5)
    jj = np.arange(1, s + 1, dtype=np.int64)[:, None]
    # sin(2πj/M)·sin(2πjk/M), and sin(πj/M)·sin(πj(2k+1)/M) for l = k+1
    diag = amp * _sin_pi_frac(2 * jj, M) * _sin_pi_frac(2 * jj * k, M)
    ku = k[:, : M - 2]
    upper = -amp * _sin_pi_frac(jj, M) * _sin_pi_frac(jj * (2 * ku + 1), M)
    A = np.concatenate([diag, upper], axis=1)
    offset = np.concatenate([np.full(M - 1, 4.0 * M), np.full(M - 2, -2.0 * M)])
    return A, offset


def fe_lognormal_coefficients(M: int, s: int) -> tuple[np.ndarray, np.ndarray]:
    """Experiment 3 (log-normal case): Θ = Ψ̂ + Y·Ψ with ψ_0 = 2 and
    ψ_j(x) = j^{-3/2} sin(2πjx) at the I = M equal-weight quadrature points,
    read as the element midpoints x_i = (i - 1/2)/M.  Returns Ψ (s x M) and
    the column offsets (all 2); a = exp(Θ)."""
    jj = np.arange(1, s + 1, dtype=np.int64)[:, None]
    i = np.arange(1, M + 1, dtype=np.int64)[None, :]
    # sin(2πj(2i-1)/(2M)) = sin(πj(2i-1)/M)
    Psi = jj.astype(np.float64) ** -1.5 * _sin_pi_frac(jj * (2 * i - 1), M)
    return Psi, np.full(M, 2.0)


def fe_workload(kind: str, N: int, M: int, s: int, seed: int = 5) -> Workload:
    """Lattice of prime N with a seeded generating vector and the inputs of
    Experiment 2 ('uniform': centred map, offsets a_0, no exp) or
    Experiment 3 ('lognormal': Φ^{-1} map, offset 2, exp)."""
    rng = np.random.default_rng(seed)
    g = PRIMITIVE_ROOT[N]
    e = rng.integers(0, N - 1, size=s)
    z = np.array([pow(g, int(v), N) for v in e], dtype=np.int64)
    if kind == "uniform":
        A, off = fe_uniform_coefficients(M, s)
        mp = "centred"
    elif kind == "lognormal":
        A, off = fe_lognormal_coefficients(M, s)
        mp = "phi_inv"
    else:
        raise ValueError(kind)
    return Workload(f"fe-{kind}-{N}-M{M}-s{s}", "prime", N, g, 0, z, False, mp, "auto",
                    A.astype(np.float32), epilogue=kind, exponents=e,
                    extra={"col_offset": off.astype(np.float32), "apply_exp": kind == "lognormal"})
