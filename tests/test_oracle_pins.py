"""Pins of the FP64 oracle against facts the paper and mathematics fix.

Each test names the passage it pins.  None of them re-types the oracle's
formula: they compare it with the printed worked example, brute force,
closed forms, library routines or an independently written computation.
"""

import json
import math
import os

import numpy as np
import pytest
import scipy.special

from oracle import circulant, f2, numtheory, points, products
from paper_1501_06286_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _example1():
    with open(os.path.join(GOLDEN, "example1_N7.json")) as f:
        return json.load(f)


# --------------------------------------------------------------------------
# Section 2.1, Example 1 (N=7, s=3, generator (1,5,3), beta=3)
# --------------------------------------------------------------------------

def test_example1_exponents_and_inverse():
    ex = _example1()
    e = numtheory.exponents(ex["generator"], ex["beta"], ex["N"])
    assert [v + 1 for v in e] == ex["c"]
    assert numtheory.inverse_mod(ex["beta"], ex["N"]) == ex["beta_inverse"]
    assert numtheory.is_primitive_root(ex["beta_inverse"], ex["N"])


def test_example1_conventional_points():
    ex = _example1()
    ps = points.PointSet("prime", ex["N"], ex["generator"], "identity", "include")
    num = ps.point_numerators(np.arange(ex["N"]))
    assert num.tolist() == ex["conventional_points_numerators"]


def test_example1_reordered_points_and_index_map():
    ex = _example1()
    N, g = ex["N"], ex["beta"]
    e = [c - 1 for c in ex["c"]]
    X = points.reordered_points_prime(N, g, e)
    assert np.array_equal(np.rint(X * N).astype(int), np.array(ex["reordered_points_numerators"][1:]))
    # conventional index of reordered point n is beta^{-(n-1)} mod N
    conv = points.reordered_conventional_index_prime(N, g)
    table = ex["conventional_points_numerators"]
    for r, n in enumerate(conv):
        assert table[n] == ex["reordered_points_numerators"][r + 1]


def test_example1_Z_and_P():
    ex = _example1()
    N, g = ex["N"], ex["beta"]
    # generator sequence numerators g^k mod N; with the identity map the
    # sequence equals numerators / N
    zeta = circulant.generator_sequence_prime(N, g, "identity")
    Z = circulant.circulant_Z(zeta)
    assert np.array_equal(np.rint(Z * N).astype(int), np.array(ex["Z_numerators"]))
    e = [c - 1 for c in ex["c"]]
    assert np.array_equal(circulant.selector_P(e, N - 1).astype(int), np.array(ex["P"]))
    # Y' = Z P (Eq. (3)) on the printed matrices
    Yp = np.array(ex["Z_numerators"]) @ np.array(ex["P"])
    assert Yp.tolist() == ex["reordered_points_numerators"][1:]


# --------------------------------------------------------------------------
# Section 2.1: primitive roots, power and log tables (brute force)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N", sorted(workloads.PRIMITIVE_ROOT))
def test_primitive_root_brute_force(N):
    g = numtheory.smallest_primitive_root(N)
    assert g == workloads.PRIMITIVE_ROOT[N]
    assert numtheory.multiplicative_order(g, N) == N - 1
    for h in range(1, g):
        assert numtheory.multiplicative_order(h, N) < N - 1
    # beta^{N-1} = 1 and beta^{-1} is primitive as well
    assert pow(g, N - 1, N) == 1
    assert numtheory.multiplicative_order(numtheory.inverse_mod(g, N), N) == N - 1


@pytest.mark.parametrize("N", [40961, 65537, 786433])
def test_primitive_root_large(N):
    g = workloads.PRIMITIVE_ROOT[N]
    assert numtheory.smallest_primitive_root(N) == g
    # order of g equals N-1: g^((N-1)/p) != 1 checked against sympy's factorisation
    sympy = pytest.importorskip("sympy")
    assert sympy.ntheory.residue_ntheory.n_order(g, N) == N - 1


def test_three_is_not_primitive_where_stated():
    for N in (7681, 12289):
        assert numtheory.multiplicative_order(3, N) < N - 1
    assert not numtheory.is_primitive_root(3, 786433)


@pytest.mark.parametrize("N", [7, 17, 257, 7681])
def test_power_log_tables(N):
    g = workloads.PRIMITIVE_ROOT[N]
    pw = numtheory.power_table(g, N)
    lg = numtheory.log_table(g, N)
    assert sorted(pw) == list(range(1, N))           # bijection onto Z_N^*
    for k in range(N - 1):
        assert pw[k] == pow(g, k, N)
        assert lg[pw[k]] == k


def test_log_table_rejects_non_primitive():
    with pytest.raises(ValueError):
        numtheory.log_table(2, 7)          # 2 has order 3 mod 7


# --------------------------------------------------------------------------
# Section 2.1, Eq. (3): Y' = Z P entry by entry, all maps, collisions included
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N", [7, 17, 257])
@pytest.mark.parametrize("phi", ["identity", "centred", "tent", "phi_inv"])
def test_circulant_identity(N, phi):
    rng = np.random.default_rng(N)
    g = workloads.PRIMITIVE_ROOT[N]
    s = 2 * N  # forces collisions
    e = rng.integers(0, N - 1, size=s)
    z = [pow(g, int(v), N) for v in e]
    ps = points.PointSet("prime", N, z, phi, "include")
    conv = points.reordered_conventional_index_prime(N, g)
    Yp = ps.Y_rows(conv)                       # rows y_1..y_{N-1}, reordered
    zeta = circulant.generator_sequence_prime(N, g, phi)
    ZP = circulant.circulant_Z(zeta) @ circulant.selector_P(e, N - 1)
    assert np.array_equal(Yp, ZP)


def test_selector_has_one_entry_per_column_and_collision_count():
    w = workloads.lattice_257()
    e = numtheory.exponents(w.gen, w.g, w.N)
    assert e == [int(v) for v in w.exponents]
    P = circulant.selector_P(e, w.N - 1)
    assert np.all(P.sum(axis=0) == 1)
    row_counts = P.sum(axis=1)
    brute_adds = int(np.sum(np.maximum(row_counts - 1, 0)))
    assert circulant.collision_adds(e) == brute_adds
    assert brute_adds == w.s - int(np.count_nonzero(row_counts))


# --------------------------------------------------------------------------
# The FFT reading of Z·a' (correlation with conj of the spectrum)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("L", [1, 2, 6, 16, 30, 256])
def test_explicit_dft_matches_numpy_fft(L):
    rng = np.random.default_rng(L)
    x = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    assert np.allclose(circulant.dft(x), np.fft.fft(x), rtol=0, atol=1e-10 * max(1, L))
    assert np.allclose(circulant.idft(np.fft.fft(x)), x, rtol=0, atol=1e-12 * max(1, L))


@pytest.mark.parametrize("N", [7, 17, 257])
def test_correlation_form_of_circulant_product(N):
    rng = np.random.default_rng(3 * N)
    g = workloads.PRIMITIVE_ROOT[N]
    zeta = circulant.generator_sequence_prime(N, g, "phi_inv")
    a = rng.standard_normal((N - 1, 3))
    Z = circulant.circulant_Z(zeta)
    got = circulant.circulant_apply_dft(zeta, a)
    assert np.allclose(got.imag, 0, atol=1e-11)
    assert np.allclose(got.real, Z @ a, rtol=0, atol=1e-11 * np.abs(Z @ a).max())
    # the transposed circulant uses DFT(zeta) without the conjugate
    Hc = circulant.dft(zeta)[:, None]
    gotT = circulant.idft(Hc * circulant.dft(a))
    assert np.allclose(gotT.real, Z.T @ a, atol=1e-11 * np.abs(Z.T @ a).max())


# --------------------------------------------------------------------------
# Dense product: brute force, row 0, closed-form column sums
# --------------------------------------------------------------------------

def test_matmul_brute_force_tiny():
    N, z = 7, [1, 5, 3]
    rng = np.random.default_rng(0)
    A = rng.standard_normal((3, 2))
    ps = points.PointSet("prime", N, z, "centred", "include")
    B = products.matmul(ps, A)
    for n in range(N):
        for k in range(2):
            acc = 0.0
            for j in range(3):
                acc += (((n * z[j]) % N) / N - 0.5) * A[j, k]
            assert abs(B[n, k] - acc) < 1e-14


@pytest.mark.parametrize("phi", ["centred", "tent", "identity"])
def test_row0_is_phi0_times_column_sum(phi):
    w = workloads.lattice_257()
    ps = points.PointSet("prime", w.N, w.gen, phi, "include")
    B0 = products.matmul_rows(ps, w.A, [0])[0]
    assert np.allclose(B0, points.phi(0.0, phi) * w.A.sum(axis=0), rtol=0, atol=1e-15)


def test_centred_column_sum_closed_form():
    # {n z/N} runs over all m/N, so sum_n ({n z/N} - 1/2) = -1/2 per coordinate:
    # sum over all N rows of B = -1/2 sum_j A_j, and 0 over rows 1..N-1.
    w = workloads.random_prime_case(257, 300, 5, seed=11, dtype=np.float64)
    ps = points.PointSet("prime", w.N, w.gen, "centred", "include")
    B = products.matmul(ps, w.A)
    assert np.allclose(B.sum(axis=0), -0.5 * w.A.sum(axis=0), atol=1e-11)
    assert np.allclose(B[1:].sum(axis=0), 0.0, atol=1e-11)


def test_phi_inv_column_sum_is_zero():
    # sum_{n=1}^{N-1} Φ^{-1}(n/N) = 0 by the symmetry Φ^{-1}(1-x) = -Φ^{-1}(x)
    w = workloads.gauss_65537(s=8, t=8)
    ps = points.PointSet("prime", w.N, w.gen, "phi_inv", "auto")
    assert ps.out_rows == w.N - 1
    B = products.matmul(ps, w.A.astype(np.float64))
    assert np.allclose(B.sum(axis=0), 0.0, atol=1e-9)


def test_gauss_cholesky_and_prefix_sum_closed_form():
    s = 64
    w = workloads.gauss_65537(s=s)
    A = w.A.astype(np.float64)
    i = np.arange(1, s + 1)
    assert np.array_equal(A.T @ A, np.minimum.outer(i, i) / s)   # Section 3.1: AᵀA = Σ
    assert np.array_equal(A, np.triu(A))
    ps = points.PointSet("prime", w.N, w.gen, "phi_inv", "auto")
    rows = np.arange(0, w.N - 1, 997)
    B = products.matmul_rows(ps, A, rows)
    Y = ps.Y_rows(ps.output_row_to_n(rows))
    assert np.allclose(B, np.cumsum(Y, axis=1) / math.sqrt(s), rtol=0, atol=1e-12)
    # Korobov exponents e_j = (j-1) d mod L, distinct (d odd)
    e = numtheory.exponents(w.gen, w.g, w.N)
    assert e == [int(v) for v in w.exponents]
    assert len(set(e)) == s


def test_ordering_does_not_change_quadrature_sum():
    w = workloads.random_prime_case(257, 40, 3, seed=5, dtype=np.float64)
    ps = points.PointSet("prime", w.N, w.gen, "centred", "include")
    B = products.matmul(ps, w.A)
    conv = points.reordered_conventional_index_prime(w.N, w.g)
    Bre = np.vstack([B[:1], B[conv]])
    f = lambda b: np.exp(np.sin(b)).sum(axis=1)
    assert abs(f(B).mean() - f(Bre).mean()) < 1e-13


def test_row_mean_equals_matvec_with_column_mean():
    w = workloads.field_786433(s=16, grid=5, dtype=np.float64)
    ps = points.PointSet("prime", w.N, w.gen, "centred", "auto")
    rows = np.arange(0, w.N, 4099)
    B = products.matmul_rows(ps, w.A, rows)
    r = products.matmul_rows(ps, w.A.mean(axis=1)[:, None], rows)[:, 0]
    assert np.allclose(products.row_mean(B), r, atol=1e-14)


def test_field_inputs_vanish_on_boundary():
    w = workloads.field_786433(s=32, grid=65, dtype=np.float64)
    A = w.A.reshape(32, 65, 65)
    assert np.all(A[:, 0, :] == 0) and np.all(A[:, 64, :] == 0)
    assert np.all(A[:, :, 0] == 0) and np.all(A[:, :, 64] == 0)
    j = 3
    x = np.arange(65) / 64
    ref = np.outer(np.sin(j * np.pi * x), np.sin(j * np.pi * x)) / j ** 2
    assert np.allclose(A[j - 1], ref, atol=1e-14)


# --------------------------------------------------------------------------
# Φ^{-1} (Section 2.1 names it; statistics.NormalDist is AS241)
# --------------------------------------------------------------------------

def test_phi_inv_against_scipy_and_textbook():
    N = 65537
    x = np.arange(1, N, 37) / N
    ours = np.array([points.phi(v, "phi_inv") for v in x])
    ref = scipy.special.ndtri(x)
    assert np.max(np.abs(ours - ref) / np.maximum(np.abs(ref), 1e-3)) < 5e-15
    assert points.phi(0.5, "phi_inv") == 0.0
    assert abs(points.phi(0.975, "phi_inv") - 1.959963984540054) < 1e-14
    assert points.phi(0.0, "phi_inv") == -math.inf
    for v in (0.01, 0.2, 0.4999):
        assert points.phi(1 - v, "phi_inv") == pytest.approx(-points.phi(v, "phi_inv"), rel=1e-14)
    assert points.phi(0.25, "tent") == 0.5 and points.phi(0.75, "tent") == 0.5
    assert points.phi(0.0, "tent") == 0.0


def test_row0_policy():
    assert points.include_row0("centred", "auto")
    assert not points.include_row0("phi_inv", "auto")
    assert points.include_row0("identity", "auto")
    assert not points.include_row0("centred", "exclude")


# --------------------------------------------------------------------------
# Remark 1: polynomial lattice rules over F_2
# --------------------------------------------------------------------------

def test_f2_textbook_primitive_polynomials():
    assert f2.is_primitive(0b10011)            # x^4 + x + 1
    assert not f2.is_primitive(0b11111)        # x^4+x^3+x^2+x+1: order 5
    assert not f2.is_primitive(0b10101)        # (x^2+x+1)^2, reducible
    assert f2.smallest_primitive(4) == 0b10011
    assert f2.smallest_primitive(3) == 0b1011  # x^3 + x + 1


def test_f2_degree16_modulus_by_brute_order():
    P = f2.smallest_primitive(16)
    # order of x by stepping until the value returns to 1
    v, k = f2.mod(2, P), 1
    while v != 1:
        v = f2.mod(v << 1, P)
        k += 1
    assert k == 65535
    # no smaller degree-16 candidate is primitive
    for Q in range((1 << 16) + 1, P, 2):
        assert not f2.is_primitive(Q)


def _digits_triangular(h, P):
    """u_k = h_{m-k} xor sum_{l<k} p_{m-k+l} u_l, from P * sum u_k x^-k = h."""
    m = f2.degree(P)
    u = []
    for k in range(1, m + 1):
        acc = (h >> (m - k)) & 1
        for l in range(1, k):
            acc ^= ((P >> (m - k + l)) & 1) & u[l - 1]
        u.append(acc)
    return u


def test_f2_digits_three_ways():
    P = f2.smallest_primitive(10)
    m = 10
    L = (1 << m) - 1
    # m-sequence of 1/P: s_i = u_1 of x^{i-1}/P (top bit of x^{i-1} mod P)
    pw = [f2.x_power(k, P) for k in range(L)]
    seq = [(pw[k] >> (m - 1)) & 1 for k in range(L)]
    vals = set()
    for k in range(L):
        long_div = f2.laurent_digits(pw[k], P)
        assert long_div == _digits_triangular(pw[k], P)
        window = [seq[(k + i) % L] for i in range(m)]
        assert long_div == window
        vals.add(f2.v_m(pw[k], P))
    assert vals == {i / (1 << m) for i in range(1, 1 << m)}


def test_f2_circulant_identity():
    m = 6
    P = f2.smallest_primitive(m)
    L = (1 << m) - 1
    rng = np.random.default_rng(6)
    e = rng.integers(0, L, size=20)
    q = [f2.x_power(int(v), P) for v in e]
    ps = points.PointSet("f2", 1 << m, q, "phi_inv", "auto", P=P)
    zeta = circulant.generator_sequence_f2(P, "phi_inv")
    ZP = circulant.circulant_Z(zeta) @ circulant.selector_P(e, L)
    # reordered row r is the point with n(x) = x^{-r} mod P
    n_of_r = [f2.x_power((L - r) % L, P) for r in range(L)]
    assert np.array_equal(ps.Y_rows(n_of_r), ZP)
    lg = f2.log_table(P)
    assert [lg[v] for v in q] == [int(v) for v in e]


def test_f2_phi_inv_column_sums_vanish():
    w = workloads.f2_65536(m=8, s=12, grid=3)
    P = f2.smallest_primitive(8)
    q = [f2.x_power_fast(int(v), P) for v in w.gen]
    ps = points.PointSet("f2", 256, q, "phi_inv", "auto", P=P)
    B = products.matmul(ps, w.A.astype(np.float64))
    assert B.shape == (255, w.t)
    assert np.allclose(B.sum(axis=0), 0.0, atol=1e-11)


# --------------------------------------------------------------------------
# Adjoint and loss gradient
# --------------------------------------------------------------------------

def test_adjoint_dot_product_identity():
    w = workloads.random_prime_case(257, 50, 4, seed=9, dtype=np.float64, map="phi_inv")
    ps = points.PointSet("prime", w.N, w.gen, "phi_inv", "auto")
    rng = np.random.default_rng(1)
    G = rng.standard_normal((ps.out_rows, 4))
    lhs = np.sum(products.matmul(ps, w.A) * G)
    rhs = np.sum(w.A * products.adjoint(ps, G))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs) + 1e-12


def test_exp_loss_gradient_finite_differences():
    w = workloads.f2_65536(m=7, s=10, grid=3)
    P = f2.smallest_primitive(7)
    q = [f2.x_power_fast(int(v), P) for v in w.gen]
    ps = points.PointSet("f2", 128, q, "phi_inv", "auto", P=P)
    A = w.A.astype(np.float64)
    loss, grad = products.exp_mean_loss_and_grad(ps, A)
    h = 1e-6
    for (j, k) in [(0, 0), (3, 4), (9, 8), (5, 2)]:
        Ap, Am = A.copy(), A.copy()
        Ap[j, k] += h
        Am[j, k] -= h
        fd = (products.exp_mean_loss(products.matmul(ps, Ap)) -
              products.exp_mean_loss(products.matmul(ps, Am))) / (2 * h)
        assert abs(fd - grad[j, k]) <= 1e-7 * max(abs(grad[j, k]), 1e-3)


# --------------------------------------------------------------------------
# Planted mistakes: each pin above must catch a plausible error
# --------------------------------------------------------------------------

def test_planted_transposed_circulant_is_caught():
    ex = _example1()
    zeta = circulant.generator_sequence_prime(7, 3, "identity")
    L = len(zeta)
    r = np.arange(L)[:, None]
    c = np.arange(L)[None, :]
    Z_wrong = zeta[(r - c) % L]
    assert not np.array_equal(np.rint(Z_wrong * 7).astype(int), np.array(ex["Z_numerators"]))


def test_planted_missing_conjugate_is_caught():
    zeta = circulant.generator_sequence_prime(17, 3, "centred")
    a = np.random.default_rng(0).standard_normal(16)
    wrong = circulant.idft(circulant.dft(zeta) * circulant.dft(a)).real
    assert not np.allclose(wrong, circulant.circulant_Z(zeta) @ a, atol=1e-8)


def test_planted_wrong_row0_is_caught():
    w = workloads.random_prime_case(17, 6, 2, seed=1, dtype=np.float64)
    ps = points.PointSet("prime", w.N, w.gen, "centred", "include")
    B = products.matmul(ps, w.A)
    B_wrong = B.copy()
    B_wrong[0] = 0.0     # forgetting y_0 a = φ(0) Σ a_j
    assert np.allclose(B.sum(axis=0), -0.5 * w.A.sum(axis=0), atol=1e-12)
    assert not np.allclose(B_wrong.sum(axis=0), -0.5 * w.A.sum(axis=0), atol=1e-12)


def test_f2_vectorised_points_match_scalar_definition():
    # the row-vectorised point construction equals the scalar one
    # (poly product mod P, then long division) entry by entry
    P = f2.smallest_primitive(7)
    rng = np.random.default_rng(3)
    q = [int(v) for v in rng.integers(1, 128, size=9)]
    ps = points.PointSet("f2", 128, q, "identity", "include", P=P)
    num = ps.point_numerators(np.arange(128))
    for n in range(128):
        for j, qj in enumerate(q):
            digits = f2.laurent_digits(f2.mulmod(n, qj, P), P)
            v = 0
            for u in digits:
                v = (v << 1) | u
            assert num[n, j] == v


# --------------------------------------------------------------------------
# Remark 2: a shift keeps Y' = Z·P only when it is the same in every
# coordinate
# --------------------------------------------------------------------------

@pytest.mark.parametrize("phi", ["centred", "phi_inv", "tent"])
def test_diagonal_shift_keeps_circulant(phi):
    # With Δ the same in every coordinate the reordered rows still factor as
    # Z·P with z_k = φ({g^k/N + Δ}); checked entry by entry at N = 17.
    N, g, delta = 17, 3, 0.3
    z = [1, 5, 3, 3, 16]
    ps = points.PointSet("prime", N, z, phi, "exclude", shift=delta)
    e = numtheory.exponents(z, g, N)
    zeta = np.array([points.phi(points.shifted(pow(g, k, N) / N, delta), phi) for k in range(N - 1)])
    Yp = circulant.circulant_Z(zeta) @ circulant.selector_P(e, N - 1)
    conv = points.reordered_conventional_index_prime(N, g)
    Y_conv = ps.Y_rows(conv)          # conventional rows g^{-r}, r = 0..N-2
    assert np.array_equal(Yp, Y_conv)


def test_diagonal_shift_row0_and_fraction():
    # row 0 is the point {0 + Δ} = Δ in every coordinate; x + Δ wraps at 1
    ps = points.PointSet("prime", 17, [1, 2], "phi_inv", "auto", shift=0.25)
    assert ps.has_row0
    assert abs(ps.phi0 - scipy.special.ndtri(0.25)) < 1e-15
    assert ps.Y_rows([0])[0, 0] == ps.phi0
    assert points.shifted(0.75, 0.25) == 0.0
    assert points.shifted(0.5, 0.25) == 0.75
    # the shifted set is the unshifted one translated mod 1
    x = ps.points(np.arange(17))
    y = ps.Y_rows(np.arange(17))
    ref = scipy.special.ndtri(np.mod(x + 0.25, 1.0))
    assert np.max(np.abs(y - ref)) < 1e-12


def test_per_coordinate_shift_breaks_circulant():
    # Remark 2: with shifts that differ between coordinates the reordered
    # rows are no longer Z·P for any one sequence z: two coordinates with
    # the same generator component (same e_j) give different columns,
    # while every column of Z·P with equal e_j is the same.
    N, g = 17, 3
    z = [5, 5]
    conv = points.reordered_conventional_index_prime(N, g)
    cols = []
    for delta in (0.1, 0.3):
        ps = points.PointSet("prime", N, [z[0]], "centred", "exclude", shift=delta)
        cols.append(ps.Y_rows(conv)[:, 0])
    assert not np.array_equal(cols[0], cols[1])
    e = numtheory.exponents(z, g, N)
    assert e[0] == e[1]
    P = circulant.selector_P(e, N - 1)
    zeta = np.random.default_rng(0).standard_normal(N - 1)
    ZP = circulant.circulant_Z(zeta) @ P
    assert np.array_equal(ZP[:, 0], ZP[:, 1])
