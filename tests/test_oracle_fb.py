"""Pins of the F_b polynomial-lattice oracle (Remark 1 over a prime base b).

What fixes it, independently of its own code:
  * b = 2: the F_b routines agree with the separate F_2 module (primitive
    polynomials, digits, whole point sets);
  * textbook primitive polynomials over F_3 (x^2 + x + 2, x^3 + 2x + 1) and
    multiplicative orders found by brute-force repeated multiplication;
  * three independent routes to the digits of h/P: the coefficient
    recurrence, the quotient of the polynomial long division h·x^m ÷ P, and
    the window of the linear recurring sequence of 1/P (the top
    coefficients of x^{k+r-1} mod P for h = x^k mod P);
  * every coordinate runs over all of {v / b^m} (closed-form column sums);
  * Y' = Z·P entry by entry under the reordering n(x) = x^{-r};
  * a planted sign mistake in the digit recurrence is caught.
"""

import numpy as np
import pytest

from oracle import circulant, f2, fb, points


def _order_brute(P, b):
    """Multiplicative order of x modulo P by repeated multiplication."""
    v = fb.divmod_poly([0, 1], P, b)[1]
    k = 1
    while v != [1]:
        v = fb.divmod_poly([0] + v, P, b)[1]
        k += 1
        if k > b ** fb.degree(P):
            return None
    return k


@pytest.mark.parametrize("m", range(2, 11))
def test_base2_agrees_with_f2_module(m):
    P = fb.smallest_primitive(m, 2)
    assert fb.encode(P, 2) == f2.smallest_primitive(m)
    Pi = f2.smallest_primitive(m)
    rng = np.random.default_rng(m)
    for h in rng.integers(0, 1 << m, size=20):
        h = int(h)
        assert fb.laurent_digits(fb.decode(h, 2, m), P, 2) == f2.laurent_digits(h, Pi)


def test_base2_point_sets_agree():
    m = 7
    Pi = f2.smallest_primitive(m)
    gen = [3, 17, 100, 1, 64]
    a = points.PointSet("f2", 1 << m, gen, "centred", "include", P=Pi).Y()
    b = points.PointSet("fb", 1 << m, gen, "centred", "include", P=Pi, base=2).Y()
    assert np.array_equal(a, b)


def test_textbook_primitive_polynomials_over_f3():
    assert fb.smallest_primitive(2, 3) == [2, 1, 1]        # x^2 + x + 2
    assert fb.smallest_primitive(3, 3) == [1, 2, 0, 1]     # x^3 + 2x + 1
    assert not fb.is_primitive([1, 0, 1], 3)               # x^2 + 1: irreducible, x has order 4
    assert _order_brute([1, 0, 1], 3) == 4
    assert not fb.is_primitive([1, 2, 1], 3)               # (x + 1)^2


@pytest.mark.parametrize("b,m", [(3, 2), (3, 3), (3, 4), (3, 5), (5, 2), (5, 3), (7, 2), (13, 2)])
def test_primitive_means_order_b_to_the_m_minus_1(b, m):
    P = fb.smallest_primitive(m, b)
    assert _order_brute(P, b) == b ** m - 1
    # every smaller monic polynomial of that degree fails the order test
    for low in range(1, fb.encode(P, b) - b ** m):
        Q = fb.decode(low, b, m) + [1]
        assert _order_brute(Q, b) != b ** m - 1


@pytest.mark.parametrize("b,m", [(3, 3), (3, 5), (5, 3), (7, 2), (11, 2)])
def test_three_digit_routes_agree(b, m):
    P = fb.smallest_primitive(m, b)
    L = b ** m - 1
    # route 3: s_j = top coefficient of x^{j-1} mod P, j >= 1
    top = []
    v = [1]
    for _ in range(L + m):
        top.append(v[m - 1] if len(v) == m else 0)
        v = fb.divmod_poly([0] + v, P, b)[1]
    for k in range(L):
        h = fb.x_power(k, P, b)
        d1 = fb.laurent_digits(h, P, b)
        q, _ = fb.divmod_poly([0] * m + h, P, b)     # h·x^m = q·P + rest
        d2 = [(q[m - r] if m - r < len(q) else 0) for r in range(1, m + 1)]
        d3 = [top[(k + r - 1) % L] for r in range(1, m + 1)]
        assert d1 == d2 == d3


def test_planted_sign_mistake_in_the_recurrence_is_caught():
    b, m = 3, 4
    P = fb.smallest_primitive(m, b)

    def wrong(h):
        hh = list(h) + [0] * (m - len(h))
        u = []
        for r in range(1, m + 1):
            acc = hh[m - r] + sum(P[m - r + k] * u[k - 1] for k in range(1, r))
            u.append(acc % b)
        return u

    caught = False
    for k in range(b ** m - 1):
        h = fb.x_power(k, P, b)
        q, _ = fb.divmod_poly([0] * m + h, P, b)
        ref = [(q[m - r] if m - r < len(q) else 0) for r in range(1, m + 1)]
        caught |= wrong(h) != ref
    assert caught


@pytest.mark.parametrize("b,m", [(3, 4), (5, 3), (7, 2)])
def test_each_coordinate_runs_over_all_points(b, m):
    P = fb.encode(fb.smallest_primitive(m, b), b)
    N = b ** m
    gen = [1, 2, N - 1, 7 % N or 1, N // 2]
    ps = points.PointSet("fb", N, gen, "identity", "include", P=P, base=b)
    num = ps.point_numerators(np.arange(N))
    for j in range(len(gen)):
        assert sorted(num[:, j].tolist()) == list(range(N))
    # closed forms: centred column sums are -1/2, Φ^{-1} sums 0 over n >= 1
    Yc = points.PointSet("fb", N, gen, "centred", "include", P=P, base=b).Y()
    assert np.allclose(Yc.sum(axis=0), -0.5, atol=1e-12)
    Yp = points.PointSet("fb", N, gen, "phi_inv", "auto", P=P, base=b).Y()
    assert Yp.shape[0] == N - 1
    assert np.allclose(Yp.sum(axis=0), 0.0, atol=1e-10)


@pytest.mark.parametrize("b,m,map", [(3, 3, "centred"), (5, 2, "phi_inv"), (3, 2, "tent"), (7, 2, "centred")])
def test_reordered_rows_factor_as_circulant_times_selector(b, m, map):
    Pc = fb.smallest_primitive(m, b)
    P = fb.encode(Pc, b)
    N = b ** m
    L = N - 1
    rng = np.random.default_rng(b * 100 + m)
    e = rng.integers(0, L, size=2 * L)      # collisions included
    gen = [fb.encode(fb.x_power(int(k), Pc, b), b) for k in e]
    ps = points.PointSet("fb", N, gen, map, "exclude", P=P, base=b)
    conv = circulant.reordered_conventional_index_fb(Pc, b)
    assert sorted(conv) == list(range(1, N))
    Yre = ps.Y_rows(np.array(conv))
    zeta = circulant.generator_sequence_fb(Pc, b, map)
    Z = circulant.circulant_Z(zeta)
    Psel = circulant.selector_P(e, L)
    assert np.array_equal(Yre, Z @ Psel)
