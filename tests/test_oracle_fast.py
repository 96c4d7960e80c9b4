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
