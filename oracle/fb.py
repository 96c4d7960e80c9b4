"""Polynomial arithmetic over F_b (b prime) for polynomial lattice rules
(oracle; test infrastructure).

Remark 1 (Section 2.1) says the fast method works in the same way for
polynomial lattice rules over a finite field; the paper gives no formulas.
This module writes the standard definition out for a prime base b, with a
monic modulus P(x) of degree m and generating polynomials q_j(x):

    n  <->  n(x) = sum_i n_i x^i   (n_i the base-b digits of n, n_0 lowest)
    x_{n,j} = v_m( n(x) q_j(x) mod P(x) / P(x) ),
    v_m( sum_{k>=1} u_k x^{-k} ) = sum_{k=1}^{m} u_k b^{-k}.

Polynomials are lists of coefficients in 0..b-1, lowest degree first; the
integer encoding used to name them is sum_i c_i b^i (a monic P of degree m
encodes as b^m + ...).  Nothing here shares code with the F_2 module; for
b = 2 the two are pinned against each other.
"""

from __future__ import annotations

from .numtheory import is_prime, prime_factors


def encode(c: list[int], b: int) -> int:
    """sum_i c_i b^i."""
    v = 0
    for d in reversed(c):
        v = v * b + d
    return v


def decode(v: int, b: int, length: int) -> list[int]:
    """The `length` lowest base-b digits of v (lowest first)."""
    out = []
    for _ in range(length):
        out.append(v % b)
        v //= b
    return out


def trim(a: list[int]) -> list[int]:
    a = list(a)
    while a and a[-1] == 0:
        a.pop()
    return a


def mul(a: list[int], c: list[int], b: int) -> list[int]:
    """Schoolbook product in F_b[x]."""
    if not a or not c:
        return []
    out = [0] * (len(a) + len(c) - 1)
    for i, ai in enumerate(a):
        if ai:
            for j, cj in enumerate(c):
                out[i + j] = (out[i + j] + ai * cj) % b
    return trim(out)


def divmod_poly(a: list[int], P: list[int], b: int) -> tuple[list[int], list[int]]:
    """Quotient and remainder of a by the monic P in F_b[x] (long division)."""
    P = trim(P)
    m = len(P) - 1
    if P[-1] != 1:
        raise ValueError("P must be monic")
    r = trim(a)
    if len(r) <= m:
        return [], r
    q = [0] * (len(r) - m)
    r = list(r)
    for k in range(len(r) - 1, m - 1, -1):
        c = r[k] % b
        if c:
            q[k - m] = c
            for i in range(m + 1):
                r[k - m + i] = (r[k - m + i] - c * P[i]) % b
    return trim(q), trim(r[:m])


def mulmod(a: list[int], c: list[int], P: list[int], b: int) -> list[int]:
    return divmod_poly(mul(a, c, b), P, b)[1]


def x_power(k: int, P: list[int], b: int) -> list[int]:
    """x^k mod P by square-and-multiply."""
    result, base = [1], divmod_poly([0, 1], P, b)[1]
    while k:
        if k & 1:
            result = mulmod(result, base, P, b)
        base = mulmod(base, base, P, b)
        k >>= 1
    return result


def degree(P: list[int]) -> int:
    return len(trim(P)) - 1


def is_primitive(P: list[int], b: int) -> bool:
    """A monic P of degree m is primitive iff x has order b^m - 1 modulo P
    (an element of that order makes F_b[x]/(P) a field, so the test also
    implies irreducibility)."""
    P = trim(P)
    m = len(P) - 1
    if m < 1 or P[-1] != 1 or P[0] == 0:
        return False
    L = b ** m - 1
    if x_power(L, P, b) != [1]:
        return False
    return all(x_power(L // p, P, b) != [1] for p in prime_factors(L)) if L > 1 else True


def smallest_primitive(m: int, b: int) -> list[int]:
    """The monic primitive polynomial of degree m over F_b with the smallest
    integer encoding."""
    if not is_prime(b):
        raise ValueError("b must be prime")
    for low in range(1, b ** m):
        P = decode(low, b, m) + [1]
        if is_primitive(P, b):
            return P
    raise ValueError(f"no primitive polynomial of degree {m} over F_{b}")


def laurent_digits(h: list[int], P: list[int], b: int) -> list[int]:
    """Digits u_1..u_m of h(x)/P(x) = sum_k u_k x^{-k}, deg h < m = deg P.

    Matching the coefficients of x^{m-r}, r = 1..m, in P(x)·sum_k u_k x^{-k}
    with those of h gives, for monic P,
        u_r = h_{m-r} - sum_{k=1}^{r-1} p_{m-r+k} u_k   (mod b).
    """
    P = trim(P)
    m = len(P) - 1
    hh = list(h) + [0] * (m - len(h))
    u = []
    for r in range(1, m + 1):
        acc = hh[m - r]
        for k in range(1, r):
            acc -= P[m - r + k] * u[k - 1]
        u.append(acc % b)
    return u


def v_m_numerator(h: list[int], P: list[int], b: int) -> int:
    """Integer v with v_m(h/P) = v / b^m."""
    v = 0
    for u in laurent_digits(h, P, b):
        v = v * b + u
    return v


def log_table(P: list[int], b: int) -> list[int]:
    """log[v] = k with x^k mod P = v (v the integer encoding), v = 1..b^m-1."""
    P = trim(P)
    m = len(P) - 1
    L = b ** m - 1
    lg = [-1] * (b ** m)
    v = [1]
    for k in range(L):
        e = encode(v, b)
        if lg[e] != -1:
            raise ValueError("P is not primitive")
        lg[e] = k
        v = divmod_poly([0] + v, P, b)[1]
    return lg
