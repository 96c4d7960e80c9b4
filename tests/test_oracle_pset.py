"""Pins of the Korobov p-set oracle (Section 2.2)."""

import numpy as np
import pytest
import scipy.special

from oracle import circulant, numtheory, points, pset


def test_pset_is_union_of_korobov_lattices():
    # block g of the conventional order is the rank-1 lattice with
    # generator (1, g, g^2, ...) (brute force with Python integers)
    K, s = 11, 4
    ps = pset.PSet(K, s, "identity")
    Y = ps.Y()
    for g in range(1, K):
        for n in range(1, K):
            row = (g - 1) * (K - 1) + (n - 1)
            assert list(Y[row] * K) == [float(n * pow(g, j) % K) for j in range(s)]


def test_pset_reordering_is_a_bijection_of_blocks():
    # Section 2.2's reordered block g (n -> β^{-(n-1)}, g -> β^{g-1}) holds
    # exactly the conventional rows of the Korobov generator β^{g-1}
    K, s, beta = 13, 5, 2
    assert numtheory.is_primitive_root(beta, K)
    ps = pset.PSet(K, s, "identity")
    binv = numtheory.inverse_mod(beta, K)
    for g in range(1, K):
        gk = pow(beta, g - 1, K)
        rows = [(gk - 1) * (K - 1) + (pow(binv, n - 1, K) - 1) for n in range(1, K)]
        assert np.array_equal(pset.reordered_block(K, s, beta, g), ps.Y_rows(rows))


@pytest.mark.parametrize("phi", ["centred", "phi_inv"])
def test_pset_blocks_factor_as_Z_P(phi):
    # Y'_g = Z·P_g with one circulant Z (z_k = φ({β^k/K})) and the exponents
    # of the c_{g,j} formula (Section 2.2), entry by entry
    K, s, beta = 17, 6, 3
    ps = pset.PSet(K, s, phi)
    zeta = circulant.generator_sequence_prime(K, beta, phi)
    Z = circulant.circulant_Z(zeta)
    binv = numtheory.inverse_mod(beta, K)
    for g in range(1, K):
        P = circulant.selector_P(pset.exponents(K, s, g), K - 1)
        gk = pow(beta, g - 1, K)
        rows = [(gk - 1) * (K - 1) + (pow(binv, n - 1, K) - 1) for n in range(1, K)]
        assert np.array_equal(Z @ P, ps.Y_rows(rows))


def test_pset_c_formula_readings_give_the_same_points():
    # c = ((j-1)(g-1) mod (K-1)) + 1 and c = (j-1)(g-1) + 1 differ as
    # integers but β^{c-n} is the same, β having order K-1
    K, beta = 19, 2
    for g in range(1, K):
        for j in range(1, 8):
            c1 = ((j - 1) * (g - 1)) % (K - 1) + 1
            c2 = (j - 1) * (g - 1) + 1
            for n in range(1, K):
                assert pow(beta, c1 - n + 10 * (K - 1), K) == pow(beta, c2 - n + 10 * (K - 1), K)


@pytest.mark.parametrize("phi", ["centred", "phi_inv"])
def test_pset_column_sums_vanish(phi):
    # for every g and j, n·g^j runs over all nonzero residues, and both the
    # centred map and Φ^{-1} sum to 0 over {v/K : v = 1..K-1}
    K, s = 31, 5
    Y = pset.PSet(K, s, phi).Y()
    assert np.max(np.abs(Y.sum(axis=0))) < 1e-9


def test_pset_matmul_against_explicit_points():
    K, s = 7, 3
    ps = pset.PSet(K, s, "phi_inv", shift=0.25)
    A = np.random.default_rng(1).standard_normal((s, 2))
    Y = np.empty((ps.out_rows, s))
    for g in range(1, K):
        for n in range(1, K):
            for j in range(s):
                x = (n * g ** j % K) / K
                Y[(g - 1) * (K - 1) + n - 1, j] = scipy.special.ndtri(points.shifted(x, 0.25))
    assert np.max(np.abs(pset.matmul(ps, A) - Y @ A)) < 1e-12
