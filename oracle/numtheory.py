"""Prime-field arithmetic for rank-1 lattice rules (oracle; test infrastructure).

Section 2.1 of the paper: N prime, Z_N^* = {1..N-1}, a primitive element
beta of Z_N^* (here ``g``), and the exponents c_j with
g_j ≡ beta^(c_j - 1) (mod N).  This module uses the 0-based exponent
e_j = c_j - 1 in [0, N-2].

Everything here is plain integer arithmetic in Python ints (exact).
"""

from __future__ import annotations


def is_prime(n: int) -> bool:
    """Trial division.  Plain and exact for the sizes used (N < 2^31)."""
    if n < 2:
        return False
    if n % 2 == 0:
        return n == 2
    d = 3
    while d * d <= n:
        if n % d == 0:
            return False
        d += 2
    return True


def prime_factors(n: int) -> list[int]:
    """Distinct prime factors of n, ascending (trial division)."""
    out = []
    d = 2
    while d * d <= n:
        if n % d == 0:
            out.append(d)
            while n % d == 0:
                n //= d
        d += 1
    if n > 1:
        out.append(n)
    return out


def multiplicative_order(g: int, N: int) -> int:
    """Smallest k >= 1 with g^k ≡ 1 (mod N), by repeated multiplication."""
    g %= N
    if g == 0:
        raise ValueError("0 has no multiplicative order")
    v, k = g, 1
    while v != 1:
        v = (v * g) % N
        k += 1
    return k


def is_primitive_root(g: int, N: int) -> bool:
    """Section 2.1: g is primitive iff {g^k mod N : k = 1..N-1} = Z_N^*.

    Equivalent test: g^((N-1)/p) != 1 for every prime p dividing N-1.
    """
    if not is_prime(N) or not (1 <= g <= N - 1):
        return False
    if N == 2:
        return g == 1
    L = N - 1
    return all(pow(g, L // p, N) != 1 for p in prime_factors(L))


def smallest_primitive_root(N: int) -> int:
    """Smallest primitive element of Z_N^* (the paper leaves beta free)."""
    for g in range(1, N):
        if is_primitive_root(g, N):
            return g
    raise ValueError(f"no primitive root mod {N}")


def power_table(g: int, N: int) -> list[int]:
    """pow[k] = g^k mod N for k = 0..N-2 (Section 2.1), by repeated
    multiplication, so that it does not reuse Python's modular pow."""
    out = [1] * (N - 1)
    v = 1
    for k in range(1, N - 1):
        v = (v * g) % N
        out[k] = v
    return out


def log_table(g: int, N: int) -> list[int]:
    """log[v] = k with g^k ≡ v (mod N), v in 1..N-1; log[0] = -1."""
    pw = power_table(g, N)
    lg = [-1] * N
    for k, v in enumerate(pw):
        if lg[v] != -1:
            raise ValueError(f"{g} is not primitive mod {N}")
        lg[v] = k
    return lg


def exponents(z, g: int, N: int) -> list[int]:
    """e_j = log_g z_j (0-based c_j - 1), Section 2.1."""
    lg = log_table(g, N)
    out = []
    for zj in z:
        v = int(zj) % N
        if v == 0:
            raise ValueError("generator component must lie in Z_N^*")
        out.append(lg[v])
    return out


def inverse_mod(a: int, N: int) -> int:
    """a^{-1} mod N for prime N (Fermat)."""
    return pow(a, N - 2, N)
