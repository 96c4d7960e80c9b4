"""Polynomial arithmetic over F_2 for polynomial lattice rules (oracle; test
infrastructure).

Remark 1 (Section 2.1) states that the method carries over to polynomial
lattice rules over a finite field; the paper gives no formulas.  This module
uses the standard definition of a polynomial lattice point set with modulus
P(x) of degree m over F_2 and generating polynomials q_j(x):

    n  <->  n(x) = sum_i n_i x^i   (n_i the binary digits of n, n_0 = LSB)
    x_{n,j} = v_m( n(x) q_j(x) / P(x) ),
    v_m( sum_{k>=1} u_k x^{-k} ) = sum_{k=1}^{m} u_k 2^{-k}.

Polynomials are Python ints: bit i is the coefficient of x^i.
"""

from __future__ import annotations

from .numtheory import prime_factors


def degree(a: int) -> int:
    return a.bit_length() - 1


def mul(a: int, b: int) -> int:
    """Carry-less product in F_2[x]."""
    out = 0
    i = 0
    while b >> i:
        if (b >> i) & 1:
            out ^= a << i
        i += 1
    return out


def mod(a: int, P: int) -> int:
    """Remainder of a modulo P in F_2[x] (schoolbook long division)."""
    m = degree(P)
    while a and degree(a) >= m:
        a ^= P << (degree(a) - m)
    return a


def mulmod(a: int, b: int, P: int) -> int:
    return mod(mul(a, b), P)


def x_power(k: int, P: int) -> int:
    """x^k mod P by k repeated multiplications by x (plain)."""
    v = 1
    for _ in range(k):
        v = mod(v << 1, P)
    return v


def x_power_fast(k: int, P: int) -> int:
    """x^k mod P by square-and-multiply (used where k is large)."""
    result, base = 1, mod(2, P)
    while k:
        if k & 1:
            result = mulmod(result, base, P)
        base = mulmod(base, base, P)
        k >>= 1
    return result


def is_primitive(P: int) -> bool:
    """P of degree m is primitive iff x has order 2^m - 1 modulo P.

    If P were reducible the unit group of F_2[x]/(P) would have fewer than
    2^m - 1 elements, so this order test also implies irreducibility.
    """
    m = degree(P)
    if m < 1 or not (P & 1):
        return False
    L = (1 << m) - 1
    if x_power_fast(L, P) != 1:
        return False
    return all(x_power_fast(L // p, P) != 1 for p in prime_factors(L)) if L > 1 else True


def smallest_primitive(m: int) -> int:
    """Smallest integer-encoded primitive polynomial of degree m."""
    for P in range((1 << m) + 1, 1 << (m + 1), 2):
        if is_primitive(P):
            return P
    raise ValueError(f"no primitive polynomial of degree {m}")


def laurent_digits(h: int, P: int) -> list[int]:
    """Digits u_1..u_m of h(x)/P(x) = sum_k u_k x^{-k}, deg h < m = deg P.

    Long division, one digit at a time: multiply the remainder by x, the
    next digit is the coefficient of x^m, subtract P if it is 1.
    """
    m = degree(P)
    r = h
    out = []
    for _ in range(m):
        r <<= 1
        u = (r >> m) & 1
        if u:
            r ^= P
        out.append(u)
    return out


def v_m(h: int, P: int) -> float:
    """v_m(h/P) = sum_{k=1}^m u_k 2^{-k}, exact in float64 for m <= 52."""
    m = degree(P)
    digits = laurent_digits(h, P)
    num = 0
    for u in digits:
        num = (num << 1) | u
    return num / float(1 << m)


def log_table(P: int) -> list[int]:
    """log[v] = k with x^k mod P = v for v in 1..2^m-1 (P primitive)."""
    m = degree(P)
    L = (1 << m) - 1
    lg = [-1] * (1 << m)
    v = 1
    for k in range(L):
        if lg[v] != -1:
            raise ValueError("P is not primitive")
        lg[v] = k
        v = mod(v << 1, P)
    return lg
