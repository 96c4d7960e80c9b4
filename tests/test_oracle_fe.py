"""Pins of the finite-element step of the oracle (oracle.fe; Sections 3.2,
3.3, Experiments 2 and 3): the constant-coefficient closed form, dense and
banded library solves, the midpoint-rule assembly element by element, and
the uniform workload's stiffness at y = 0."""

import numpy as np
import pytest

from oracle import fe
from paper_1501_06286_gb300 import workloads


@pytest.mark.parametrize("M", [3, 4, 17, 200])
@pytest.mark.parametrize("a", [2.0, np.exp(2.0)])
def test_constant_coefficient_is_nodally_exact(M, a):
    # tridiag rows: diag 2aM, off -aM (the stiffness of a ≡ a); midpoint
    # rows: a at every element midpoint
    row_t = np.concatenate([np.full(M - 1, 2 * a * M), np.full(M - 2, -a * M)])
    row_m = np.full(M, a)
    exact = fe.constant_coefficient_solution(M, a)
    for row, kind in [(row_t, "tridiag"), (row_m, "midpoint")]:
        u = fe.mean_solution(row[None, :], M, kind)
        assert np.max(np.abs(u - exact)) <= 1e-10 * np.max(exact)


def test_uniform_offsets_give_the_a_equal_two_solution():
    # Experiment 2 at y = 0: B = a_0 (diag 4M, off -2M), a ≡ 2
    M = 50
    _, off = workloads.fe_uniform_coefficients(M, 5)
    u = fe.mean_solution(off[None, :].astype(np.float64), M, "tridiag")
    assert np.max(np.abs(u - fe.constant_coefficient_solution(M, 2.0))) <= 1e-10


def test_solve_matches_dense_and_banded_solves():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(1)
    M, rows = 40, 6
    off = -rng.uniform(0.5, 1.5, size=(rows, M - 2))
    diag = np.abs(np.pad(off, ((0, 0), (1, 0)))) + np.abs(np.pad(off, ((0, 0), (0, 1)))) + rng.uniform(0.1, 1, (rows, M - 1))
    rhs = rng.standard_normal(M - 1)
    u = fe.solve_tridiag(diag, off, rhs)
    for r in range(rows):
        K = np.diag(diag[r]) + np.diag(off[r], 1) + np.diag(off[r], -1)
        assert np.allclose(u[r], np.linalg.solve(K, rhs), rtol=1e-12, atol=1e-12)
        ab = np.zeros((3, M - 1))
        ab[0, 1:], ab[1], ab[2, :-1] = off[r], diag[r], off[r]
        assert np.allclose(u[r], scipy_linalg.solve_banded((1, 1), ab, rhs), rtol=1e-12, atol=1e-12)


def test_midpoint_assembly_element_by_element():
    # assemble from the element stiffness M·a_i·[[1, -1], [-1, 1]] over the
    # M elements, keep the interior nodes 1..M-1
    rng = np.random.default_rng(2)
    M = 12
    a = rng.uniform(0.5, 3.0, size=M)
    K = np.zeros((M + 1, M + 1))
    for i in range(1, M + 1):                      # element i = [x_{i-1}, x_i]
        K[np.ix_([i - 1, i], [i - 1, i])] += M * a[i - 1] * np.array([[1.0, -1.0], [-1.0, 1.0]])
    Kint = K[1:M, 1:M]
    diag, off = fe.stiffness(a[None, :], M, "midpoint")
    assert np.allclose(diag[0], np.diag(Kint)) and np.allclose(off[0], np.diag(Kint, 1))


def test_mean_is_the_mean_of_the_solutions():
    rng = np.random.default_rng(3)
    M = 9
    a = rng.uniform(1, 2, size=(5, M))
    u_each = [fe.mean_solution(a[i:i + 1], M, "midpoint") for i in range(5)]
    assert np.allclose(fe.mean_solution(a, M, "midpoint"), np.mean(u_each, axis=0), rtol=1e-14)
