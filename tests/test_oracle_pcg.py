"""Pins of the oracle's preconditioned conjugate gradients (symmetric
Gauss-Seidel preconditioner from the lower triangle, or the IC(0) factor)
against a dense solve, the dense preconditioner inverse, CG's finite
termination, numpy's Cholesky factor where IC(0) drops no fill, and IC(0)'s
defining property."""
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


def tridiagonal_spd(n, seed):
    """1D Laplacian with a jittered diagonal: no Cholesky fill."""
    d = 2.0 + np.random.default_rng(seed).uniform(0, 0.5, n)
    rows, cols, vals = [], [], []
    for i in range(n):
        if i:
            rows.append(i); cols.append(i - 1); vals.append(-1.0)
        rows.append(i); cols.append(i); vals.append(d[i])
    M = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    return mg.CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data)


def test_ic0_is_the_cholesky_factor_without_fill():
    # tridiagonal: the exact Cholesky factor has the pattern of the lower
    # triangle, so IC(0) is it
    A = mg.symmetric_from_lower(tridiagonal_spd(50, 1))
    C = opcg.ic0(opcg.lower_triangle(A))
    ref = np.linalg.cholesky(dense(A))
    assert np.allclose(dense(C), ref, rtol=0, atol=1e-14)
    # a dense pattern: again no fill
    n = 12
    G = np.random.default_rng(2).standard_normal((n, n))
    S = G @ G.T + n * np.eye(n)
    T = sp.csr_matrix(np.tril(S))
    Lo = mg.CSR(n, T.indptr.astype(np.int32), T.indices.astype(np.int32), T.data)
    C = opcg.ic0(Lo)
    assert np.allclose(dense(C), np.linalg.cholesky(S), rtol=0, atol=1e-12)


@pytest.mark.parametrize("make", [lambda: mg.stencil2d(9), lambda: mg.stencil3d(5, seed=8),
                                  lambda: mg.random_lower(40, seed=9, density=0.2,
                                                          diag_min=4.0)])
def test_ic0_matches_a_on_its_pattern(make):
    L = make()
    A = mg.symmetric_from_lower(L)
    C = opcg.ic0(opcg.lower_triangle(A))
    assert np.array_equal(C.row_ptr, L.row_ptr) and np.array_equal(C.col, L.col)
    P = dense(C) @ dense(C).T
    Ad = dense(A)
    mask = dense(mg.CSR(L.n, L.row_ptr, L.col, np.ones_like(L.val))) != 0
    assert np.allclose(P[mask], Ad[mask], rtol=0, atol=1e-12 * np.abs(Ad).max())
    # off the pattern the product differs: IC(0) drops the fill
    assert not np.allclose(P, Ad, rtol=0, atol=1e-12)


def test_ic0_breakdown_raises():
    # symmetric but indefinite: the second pivot is 1 - 4 < 0
    Lo = mg.CSR(2, np.array([0, 1, 3], np.int32), np.array([0, 0, 1], np.int32),
                np.array([1.0, 2.0, 1.0]))
    with pytest.raises(ValueError):
        opcg.ic0(Lo)


def test_pcg_with_exact_ic0_converges_in_one_step():
    A = mg.symmetric_from_lower(tridiagonal_spd(64, 3))
    b = mg.rhs_uniform(A.n, seed=4)
    x, it, rel = opcg.pcg(A, b, np.zeros(A.n), rtol=1e-12, max_iter=10, precond="ic0")
    assert it == 1 and rel <= 1e-12


def test_pcg_ic0_reaches_the_dense_solution():
    A = mg.symmetric_from_lower(mg.stencil3d(6, seed=3))
    b = mg.rhs_uniform(A.n, seed=5)
    x, it, rel = opcg.pcg(A, b, np.zeros(A.n), rtol=1e-13, max_iter=500, precond="ic0")
    assert rel <= 1e-13
    assert oracle.relerr(x, np.linalg.solve(dense(A), b)) <= 1e-11
