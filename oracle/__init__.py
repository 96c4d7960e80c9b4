"""FP64 CPU oracle for the fast QMC matrix product B = Y·A.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library
and its Python binding) may import, call or link anything in this package.
Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.

The oracle is written from Dick, Kuo, Le Gia, Schwab, "Fast QMC
matrix-vector multiplication" (arXiv 1501.06286) and shares no code with the
GPU path.  It computes the *definition* of the product: it materialises the
lattice points {n·z_j/N} (Section 2.1) or the polynomial-lattice points
v_m(n(x)q_j(x)/P(x)) (Remark 1), applies the coordinate map φ (Section 2.1)
and multiplies densely in float64.  The circulant factorisation Y' = Z·P
(Section 2.1, Eq. (3)) is written out here only so that tests can pin it
against the dense definition, entry by entry.

Modules
-------
numtheory  prime-field arithmetic: primality, primitive roots, power and
           discrete-log tables (Section 2.1).
f2         polynomial arithmetic over F_2, primitive polynomials and the
           digit expansion v_m (Remark 1).
fb         the same over F_b for a prime base b (Remark 1), written
           independently of f2 and pinned against it at b = 2.
points     point sets in conventional and reordered order, maps φ
           (Section 2.1).
circulant  generator sequence z_k, circulant Z, selector P, explicit DFT
           (Section 2.1).
products   dense Y·A, the adjoint Yᵀ·G, the row mean and the exp-mean loss
           (Sections 1, 3.1–3.3).
fe         the finite-element step of Sections 3.2, 3.3 (Experiments 2, 3):
           tridiagonal stiffness matrices from the product's rows, their
           solves and the mean of the solutions.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against a fact the paper or mathematics fixes (the worked Example 1,
brute force, closed-form column sums, the Cholesky identity, finite
differences, two independent F_2 digit computations, three independent
F_b digit computations).  The paper prints no
error bound for the fast product, so the FP32 tolerance is a stated target,
not a pin.
"""

from . import numtheory, f2, fb, points, circulant, products, fe  # noqa: F401
