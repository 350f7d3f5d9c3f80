"""Pins of the oracle's forward substitution (Sec. II, Algorithm 1) against
facts that do not come from the oracle itself: closed forms, exact rational
solves by a different algorithm (sympy LU), scipy's triangular solver,
manufactured solutions and the backward-error bound of forward substitution.
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import matgen as mg
import oracle

EPS = np.finfo(np.float64).eps


def to_scipy(A):
    return sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n))


def test_identity_is_exact():
    n = 257
    A = mg.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32),
               np.ones(n))
    b = mg.rhs_uniform(n, seed=1)
    assert np.array_equal(oracle.forward_subst(A, b), b)


def test_diagonal_is_correctly_rounded_quotient():
    n = 500
    rng = np.random.default_rng(3)
    d = rng.uniform(0.1, 10.0, n) * rng.choice([-1, 1], n)
    A = mg.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d)
    b = rng.standard_normal(n)
    assert np.array_equal(oracle.forward_subst(A, b), b / d)


def test_unit_bidiagonal_counts_up():
    # x_i - x_{i-1} = 1, x_0 = 1  =>  x_i = i + 1 exactly
    n = 1000
    A = mg.chain(n, a=1.0, diag=1.0)
    x = oracle.forward_subst(A, np.ones(n))
    assert np.array_equal(x, np.arange(1, n + 1, dtype=np.float64))


def test_general_bidiagonal_closed_form():
    # d x_i - a x_{i-1} = b_i  =>  x_i = sum_k a^(i-k) b_k / d^(i-k+1),
    # exact in binary floating point for d = 2, a = 1 and small integer b.
    n = 40
    A = mg.chain(n, a=1.0, diag=2.0)
    rng = np.random.default_rng(5)
    b = rng.integers(-8, 9, n).astype(np.float64)
    x = oracle.forward_subst(A, b)
    for i in range(n):
        exact = sum(Fraction(int(b[k])) / Fraction(2) ** (i - k + 1)
                    for k in range(i + 1))
        assert Fraction(x[i]) == exact


@pytest.mark.parametrize("seed", range(6))
def test_exact_rational_lu_solve(seed):
    sympy = pytest.importorskip("sympy")
    n = 4 + seed
    A = mg.random_lower(n, seed=100 + seed, density=0.6, integer=True)
    dense = to_scipy(A).toarray()
    rng = np.random.default_rng(seed)
    b = rng.integers(-5, 6, n).astype(np.float64)
    M = sympy.Matrix([[sympy.Rational(int(v)) for v in row] for row in dense])
    exact = M.LUsolve(sympy.Matrix([sympy.Rational(int(v)) for v in b]))
    x = oracle.forward_subst(A, b)
    for i in range(n):
        e = Fraction(int(exact[i].p), int(exact[i].q))
        assert abs(Fraction(x[i]) - e) <= abs(e) * Fraction(4 * n) * Fraction(EPS) + Fraction(1, 10**300)


@pytest.mark.parametrize("seed", range(4))
def test_matches_scipy_triangular_solver(seed):
    A = mg.random_lower(300, seed=seed, density=0.05)
    b = mg.rhs_uniform(300, nrhs=3, seed=seed)
    x = oracle.forward_subst(A, b)
    ref = spla.spsolve_triangular(to_scipy(A), b, lower=True)
    assert oracle.relerr(x, ref) < 1e-13


def test_manufactured_solution_stencil2d():
    A = mg.stencil2d(64)
    rng = np.random.default_rng(1000)
    x_true = rng.uniform(-1, 1, A.n)
    b = mg.manufactured_rhs(A, x_true)
    assert oracle.relerr(oracle.forward_subst(A, b), x_true) < 1e-13


@pytest.mark.parametrize("cfg", [1, 2, 3])
def test_backward_error_bound(cfg):
    # forward substitution is backward stable: |b - L x| <= c n_row eps |L||x|
    A = mg.config_matrix(cfg, small=True)
    b = mg.rhs_uniform(A.n, seed=cfg)
    x = oracle.forward_subst(A, b)
    S = to_scipy(A)
    r = b - S @ x
    scale = abs(S) @ np.abs(x) + np.abs(b)
    row_len = np.diff(A.row_ptr)
    assert np.all(np.abs(r) <= 2 * row_len * EPS * scale)
    norm = np.abs(r).max() / (spla.norm(S, np.inf) * np.abs(x).max() + np.abs(b).max())
    assert norm < 10 * EPS


def test_multi_rhs_columns_are_independent_solves():
    A = mg.config_matrix(3, small=True)
    B = mg.rhs_uniform(A.n, nrhs=5, seed=9)
    X = oracle.forward_subst(A, B)
    for c in range(5):
        assert np.array_equal(X[:, c], oracle.forward_subst(A, B[:, c].copy()))


def test_residual_matches_scipy():
    A = mg.config_matrix(3, small=True)
    x = mg.rhs_uniform(A.n, nrhs=2, seed=4)
    b = mg.rhs_uniform(A.n, nrhs=2, seed=5)
    r = oracle.residual(A, x, b)
    assert np.allclose(r, b - to_scipy(A) @ x, rtol=0, atol=1e-14)


def test_invalid_inputs_rejected():
    A = mg.chain(4)
    bad = mg.CSR(4, A.row_ptr.copy(), A.col.copy(), A.val.copy())
    bad.val[-1] = 0.0
    with pytest.raises(ValueError, match="zero diagonal"):
        oracle.forward_subst(bad, np.ones(4))
    nodiag = mg.CSR(2, np.array([0, 1, 2], np.int32), np.array([0, 0], np.int32),
                    np.ones(2))
    with pytest.raises(ValueError, match="missing diagonal"):
        oracle.forward_subst(nodiag, np.ones(2))
    upper = mg.CSR(2, np.array([0, 2, 3], np.int32), np.array([0, 1, 1], np.int32),
                   np.ones(3))
    with pytest.raises(ValueError, match="wrong side of the diagonal"):
        oracle.forward_subst(upper, np.ones(2))
