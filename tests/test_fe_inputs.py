"""The applications' inputs (Sections 3.2, 3.3; Experiments 2, 3) against
numerical quadrature of their defining integrals (an independent route to
the printed closed forms)."""

import numpy as np
import pytest
from scipy import integrate

from paper_1501_06286_gb300 import workloads


def _hat_slope(k, M, x):
    """φ'_k(x) for the hat function at x_k = k/M (support [x_{k-1}, x_{k+1}])."""
    if (k - 1) / M <= x <= k / M:
        return M
    if k / M <= x <= (k + 1) / M:
        return -M
    return 0.0


@pytest.mark.parametrize("M,s", [(7, 5), (12, 3)])
def test_uniform_stiffness_coefficients_by_quadrature(M, s):
    A, off = workloads.fe_uniform_coefficients(M, s)
    assert A.shape == (s, 2 * M - 3) and off.shape == (2 * M - 3,)
    for j in range(1, s + 1):
        psi = lambda x: j ** -1.5 * np.sin(2 * np.pi * j * x)
        for k in range(1, M):
            # a_{j,k,k} = ∫ ψ_j (φ'_k)^2 over the two elements of the support
            val = sum(integrate.quad(lambda x: psi(x) * M * M, a / M, (a + 1) / M, epsabs=1e-13)[0]
                      for a in (k - 1, k))
            assert abs(A[j - 1, k - 1] - val) <= 1e-9 * max(1.0, abs(val))
            if k < M - 1:
                # a_{j,k,k+1} = ∫ ψ_j φ'_k φ'_{k+1} over [x_k, x_{k+1}]
                val = integrate.quad(lambda x: psi(x) * (-M) * M, k / M, (k + 1) / M, epsabs=1e-13)[0]
                assert abs(A[j - 1, M - 1 + k - 1] - val) <= 1e-9 * max(1.0, abs(val))
    # a_0 from ψ_0 = 2: 2·∫ φ'_k φ'_l
    for k in range(1, M):
        d = integrate.quad(lambda x: 2 * _hat_slope(k, M, x) ** 2, (k - 1) / M, (k + 1) / M,
                           points=[k / M])[0]
        assert abs(off[k - 1] - d) <= 1e-9 * d
    assert np.all(off[M - 1:] == -2.0 * M)


def test_lognormal_field_at_midpoints():
    M, s = 9, 6
    Psi, off = workloads.fe_lognormal_coefficients(M, s)
    x = (np.arange(1, M + 1) - 0.5) / M
    ref = np.array([[j ** -1.5 * np.sin(2 * np.pi * j * xi) for xi in x] for j in range(1, s + 1)])
    assert np.max(np.abs(Psi - ref)) < 1e-14
    assert np.all(off == 2.0)
