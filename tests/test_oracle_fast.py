"""The CPU form of the fast product (oracle.fast) against the dense oracle.

The two compute B = Y·A by different routes: ``products`` materialises the
points from their definition ({n z_j/N}; F_2 long division) and multiplies,
``fast`` follows Section 2.1 (exponents, scatter-add, FFT correlation with
the generator sequence, un-permute).  Agreement to FP64 round-off pins the
circulant reading, the row maps and the row-0 policy of the fast form.
"""

import numpy as np
import pytest

from oracle import f2, fast, numtheory, points, products


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b))))


@pytest.mark.parametrize("N", [7, 17, 257, 7681])
@pytest.mark.parametrize("phi", ["identity", "centred", "tent", "phi_inv"])
def test_fast_prime_matches_dense(N, phi):
    rng = np.random.default_rng(N)
    s = 40 if N > 17 else 5
    z = rng.integers(1, N, size=s)       # collisions included when N is small
    ps = points.PointSet("prime", N, z, phi)
    A = rng.standard_normal((s, 3))
    B = fast.matmul_fft(ps, A)
    ref = products.matmul(ps, A)
    assert B.shape == ref.shape
    assert _rel(B, ref) < 1e-12


@pytest.mark.parametrize("row0", ["include", "exclude"])
def test_fast_row0_policy(row0):
    N = 257
    rng = np.random.default_rng(3)
    ps = points.PointSet("prime", N, rng.integers(1, N, size=12), "centred", row0=row0)
    A = rng.standard_normal((12, 2))
    B = fast.matmul_fft(ps, A, g=numtheory.smallest_primitive_root(N))
    ref = products.matmul(ps, A)
    assert B.shape[0] == (N if row0 == "include" else N - 1)
    assert _rel(B, ref) < 1e-12


def test_fast_other_primitive_root():
    # the result does not depend on which primitive root orders the rows
    N = 257
    rng = np.random.default_rng(5)
    ps = points.PointSet("prime", N, rng.integers(1, N, size=9), "tent")
    A = rng.standard_normal((9, 2))
    roots = [g for g in range(2, 40) if numtheory.is_primitive_root(g, N)][:3]
    outs = [fast.matmul_fft(ps, A, g=g) for g in roots]
    for B in outs[1:]:
        assert _rel(B, outs[0]) < 1e-12


@pytest.mark.parametrize("m", [4, 6, 8])
@pytest.mark.parametrize("phi", ["centred", "phi_inv"])
def test_fast_f2_matches_dense(m, phi):
    P = f2.smallest_primitive(m)
    rng = np.random.default_rng(m)
    s = 7
    q = [int(v) for v in rng.integers(1, 1 << m, size=s)]
    ps = points.PointSet("f2", 1 << m, q, phi, P=P)
    A = rng.standard_normal((s, 4))
    assert _rel(fast.matmul_fft(ps, A), products.matmul(ps, A)) < 1e-12


def test_fast_plan_reuse_and_vector():
    N = 17
    ps = points.PointSet("prime", N, [1, 5, 3, 3], "centred")
    plan = fast.FastPlan(ps)
    a = np.array([0.5, -1.0, 2.0, 0.25])
    b = plan.matmul(a)
    assert b.shape == (N, 1)
    assert _rel(b[:, 0], products.matmul(ps, a[:, None])[:, 0]) < 1e-12
    # a planted mistake in the fast form (DFT of ζ without the conjugate,
    # i.e. the transposed circulant) is caught by the dense product
    bad = fast.FastPlan(ps)
    bad.spec = np.conj(bad.spec)
    assert _rel(bad.matmul(a), products.matmul(ps, a[:, None])) > 1e-3


@pytest.mark.parametrize("kind", ["prime", "f2"])
@pytest.mark.parametrize("phi", ["centred", "phi_inv"])
def test_fast_diagonal_shift(kind, phi):
    rng = np.random.default_rng(11)
    if kind == "prime":
        ps = points.PointSet("prime", 257, rng.integers(1, 257, size=20), phi, shift=0.3717)
    else:
        P = f2.smallest_primitive(7)
        ps = points.PointSet("f2", 128, [int(v) for v in rng.integers(1, 128, size=9)], phi, P=P,
                             shift=0.3717)
    assert ps.has_row0   # φ(Δ) is finite for Δ in (0, 1)
    A = rng.standard_normal((ps.s, 3))
    assert _rel(fast.matmul_fft(ps, A), products.matmul(ps, A)) < 1e-12


@pytest.mark.parametrize("L1,L2,s", [(30, 256, 40), (160, 256, 700), (768, 1024, 2048)])
def test_first_pass_as_sums_over_the_rows_of_a_line(L1, L2, s):
    """The identity behind the library's sparse first pass and its
    term-by-term first-pass lines (four-step DFT of P·A, Section 2.1): with
    positions e_j = n1_j·L2 + n2_j, the first pass's output on line k1,
    point n2 is Σ_{j: n2_j = n2} a_j·w_L1^{-(n1_j·k1 mod L1)}·w_L^{-n2·k1},
    and the L2-point DFT of line k1 over n2 gives the length-L DFT of P·a at
    index k1 + L1·k2.  Checked against numpy's FFT of the scattered vector."""
    L = L1 * L2
    rng = np.random.default_rng(L)
    e = rng.integers(0, L, size=s)
    e[1] = e[0]                                   # a collision
    a = rng.standard_normal(s) + 1j * rng.standard_normal(s)
    x = np.zeros(L, dtype=complex)
    np.add.at(x, e, a)                            # P·a
    n1, n2 = e // L2, e % L2
    k1 = np.arange(L1)[:, None]
    F = np.zeros((L1, L2), dtype=complex)
    # sums over the rows of each line, in exact integer exponents
    w1 = np.exp(-2j * np.pi * ((n1[None, :] * k1) % L1) / L1)
    w2 = np.exp(-2j * np.pi * ((n2[None, :] * k1) % L) / L)
    for col in range(L1):
        np.add.at(F[col], n2, a * w1[col] * w2[col])
    # the same first pass as a length-L1 transform of each line
    lines = x.reshape(L1, L2)                     # lines[n1, n2] = x[n1·L2 + n2]
    Fd = np.fft.fft(lines, axis=0) * np.exp(-2j * np.pi * ((np.arange(L2)[None, :] * k1) % L) / L)
    assert np.max(np.abs(F - Fd)) <= 1e-9 * np.max(np.abs(Fd))
    # second pass: X[k1 + L1·k2] = DFT_L2 over n2 of line k1
    X = np.fft.fft(F, axis=1)
    ref = np.fft.fft(x)
    idx = np.arange(L1)[:, None] + L1 * np.arange(L2)[None, :]
    assert np.max(np.abs(X - ref[idx])) <= 1e-9 * np.max(np.abs(ref))
