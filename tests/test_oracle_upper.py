"""Pins of the oracle's backward substitution (an upper triangle, rows from
the last to the first) and of its operator helpers (A^T, op(A) x = b)
against facts that do not come from the oracle: closed forms, exact
rational solves (sympy), scipy's triangular solver, dense transposes and
the backward-error bound."""
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


def upper_chain(n, a, diag):
    """diag on the diagonal, -a right of it."""
    return mg.transposed(mg.chain(n, a=a, diag=diag))


def test_identity_and_diagonal_are_exact():
    n = 300
    rng = np.random.default_rng(2)
    d = rng.uniform(0.1, 10.0, n) * rng.choice([-1, 1], n)
    D = mg.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d)
    b = rng.standard_normal(n)
    assert np.array_equal(oracle.backward_subst(D, b), b / d)


def test_unit_upper_bidiagonal_counts_down():
    # x_i - x_{i+1} = 1, x_{n-1} = 1  =>  x_i = n - i exactly
    n = 1000
    x = oracle.backward_subst(upper_chain(n, 1.0, 1.0), np.ones(n))
    assert np.array_equal(x, np.arange(n, 0, -1, dtype=np.float64))


def test_upper_bidiagonal_geometric_closed_form():
    # x_i = 1 + x_{i+1} / 2  =>  x_i = 2 - 2^-(n-1-i), exact while n - i <= 53
    n = 50
    x = oracle.backward_subst(upper_chain(n, 0.5, 1.0), np.ones(n))
    for i in range(n):
        assert Fraction(x[i]) == 2 - Fraction(1, 2 ** (n - 1 - i))


@pytest.mark.parametrize("seed", range(5))
def test_exact_rational_solve(seed):
    sympy = pytest.importorskip("sympy")
    n = 4 + seed
    U = mg.transposed(mg.random_lower(n, seed=200 + seed, density=0.6, integer=True))
    dense = to_scipy(U).toarray()
    assert np.allclose(dense, np.triu(dense))
    rng = np.random.default_rng(seed)
    b = rng.integers(-5, 6, n).astype(np.float64)
    M = sympy.Matrix([[sympy.Rational(int(v)) for v in row] for row in dense])
    exact = M.LUsolve(sympy.Matrix([sympy.Rational(int(v)) for v in b]))
    x = oracle.backward_subst(U, b)
    for i in range(n):
        e = Fraction(int(exact[i].p), int(exact[i].q))
        assert abs(Fraction(x[i]) - e) <= abs(e) * Fraction(4 * n) * Fraction(EPS) + Fraction(1, 10**300)


@pytest.mark.parametrize("seed", range(3))
def test_matches_scipy_upper_solver(seed):
    U = mg.transposed(mg.random_lower(300, seed=seed, density=0.05))
    b = mg.rhs_uniform(300, nrhs=3, seed=seed)
    ref = spla.spsolve_triangular(to_scipy(U), b, lower=False)
    assert oracle.relerr(oracle.backward_subst(U, b), ref) < 1e-13


def test_backward_error_bound():
    U = mg.transposed(mg.config_matrix(3, small=True))
    b = mg.rhs_uniform(U.n, seed=3)
    x = oracle.backward_subst(U, b)
    S = to_scipy(U)
    r = b - S @ x
    scale = abs(S) @ np.abs(x) + np.abs(b)
    assert np.all(np.abs(r) <= 2 * np.diff(U.row_ptr) * EPS * scale)


def test_transpose_matches_dense_and_is_an_involution():
    A = mg.random_lower(60, seed=4, density=0.2)
    T = oracle.transpose(A)
    assert np.array_equal(to_scipy(T).toarray(), to_scipy(A).toarray().T)
    TT = oracle.transpose(T)
    assert np.array_equal(TT.row_ptr, A.row_ptr) and np.array_equal(TT.col, A.col)
    assert np.array_equal(TT.val, A.val)
    G = mg.transposed(A)  # the input generator's own rearrangement agrees
    assert np.array_equal(G.row_ptr, T.row_ptr) and np.array_equal(G.col, T.col)
    assert np.array_equal(G.val, T.val)


@pytest.mark.parametrize("op", [0, 1, 2, 3])
def test_solve_op_satisfies_its_equation(op):
    L = mg.random_lower(200, seed=7, density=0.05)
    A = L if op in (0, 2) else mg.transposed(L)   # lower for 0/2, upper for 1/3
    D = to_scipy(A).toarray()
    M = D if op in (0, 1) else D.T
    b = mg.rhs_uniform(200, nrhs=2, seed=op)
    x = oracle.solve_op(A, b, op)
    r = b - M @ x
    assert np.abs(r).max() <= 50 * EPS * (np.abs(M).sum(1).max() * np.abs(x).max() + 1)


def test_invalid_upper_inputs_rejected():
    L = mg.chain(4)
    with pytest.raises(ValueError, match="wrong side"):
        oracle.backward_subst(L, np.ones(4))
    U = upper_chain(4, 1.0, 1.0)
    bad = mg.CSR(4, U.row_ptr.copy(), U.col.copy(), U.val.copy())
    bad.val[0] = 0.0
    with pytest.raises(ValueError, match="zero diagonal"):
        oracle.backward_subst(bad, np.ones(4))
