"""Pins of the oracle's preconditioned conjugate gradients (symmetric
Gauss-Seidel preconditioner from the lower triangle) against a dense solve,
the dense preconditioner inverse, and CG's finite termination."""
import numpy as np
import pytest
import scipy.sparse as sp

import matgen as mg
import oracle
from oracle import pcg as opcg


def dense(A):
    return sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n)).toarray()


def test_symmetric_from_lower_is_symmetric_with_that_lower_triangle():
    L = mg.stencil3d(5, seed=1)
    A = mg.symmetric_from_lower(L)
    D = dense(A)
    assert np.array_equal(D, D.T)
    assert np.array_equal(np.tril(D), dense(L))
    Lo = opcg.lower_triangle(A)
    assert np.array_equal(Lo.row_ptr, L.row_ptr) and np.array_equal(Lo.col, L.col)


def test_sgs_apply_is_the_inverse_of_the_dense_preconditioner():
    A = mg.symmetric_from_lower(mg.stencil2d(7))
    D = dense(A)
    Lo = np.tril(D)
    M = Lo @ np.diag(1.0 / np.diag(D)) @ Lo.T
    r = mg.rhs_uniform(A.n, seed=2)
    z = opcg.sgs_apply(opcg.lower_triangle(A), r)
    assert np.allclose(M @ z, r, rtol=0, atol=1e-12 * np.abs(r).max())


@pytest.mark.parametrize("make", [lambda: mg.stencil2d(12), lambda: mg.stencil3d(6, seed=3)])
def test_pcg_reaches_the_dense_solution(make):
    A = mg.symmetric_from_lower(make())
    b = mg.rhs_uniform(A.n, seed=4)
    x, it, rel = opcg.pcg(A, b, np.zeros(A.n), rtol=1e-13, max_iter=500)
    ref = np.linalg.solve(dense(A), b)
    assert rel <= 1e-13
    assert oracle.relerr(x, ref) <= 1e-11


def test_cg_terminates_within_n_steps():
    # a small SPD system: CG (any SPD preconditioner) reaches the solution in
    # at most n steps in exact arithmetic; allow two for rounding
    n = 24
    L = mg.random_lower(n, seed=5, density=0.3, diag_min=3.0)
    A = mg.symmetric_from_lower(L)
    D = dense(A)
    assert np.all(np.linalg.eigvalsh(D) > 0)
    b = mg.rhs_uniform(n, seed=6)
    x, it, rel = opcg.pcg(A, b, np.zeros(n), rtol=1e-12, max_iter=10 * n)
    assert it <= n + 2 and rel <= 1e-12
    assert oracle.relerr(x, np.linalg.solve(D, b)) <= 1e-9
