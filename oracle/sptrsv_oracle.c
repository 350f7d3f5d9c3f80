/*
 * CPU oracle for the sparse lower-triangular solve (test infrastructure).
 *
 * This file is test infrastructure only: the tests, the smoke check and the
 * CPU-baseline leg of the benchmark call it; the library's own code path never
 * does.  It shares no code, header or table with the CUDA implementation.
 *
 * Everything here is the plain definition, written out serially in FP64:
 *   - oracle_forward_subst: the serial CSR forward substitution of the
 *     paper's Section II (Fig. 1, Algorithm 1): for each row, the inner loop
 *     subtracts the products of the row's off-diagonal nonzeros with the
 *     already-solved unknowns, then the sum is divided by the diagonal.
 *   - oracle_levels: the level of each row in the dependency graph DAG_L of
 *     Section II (row i depends on row j when L[i][j] is stored, j < i): the
 *     longest dependency path that ends at the row, sources at level 0.
 *   - oracle_spmv_lower: r = b - L x, the residual used by the refinement
 *     checks.
 *   - oracle_backward_subst: the same substitution for an upper-triangular
 *     matrix, rows visited from the last to the first (the mirror image of
 *     Algorithm 1: row i needs the unknowns of rows j > i).
 *
 * CSR convention: row_ptr[n+1], col[nnz] ascending inside each row,
 * val[nnz]; every row stores its diagonal.  Right-hand sides and solutions
 * are row-major [n][nrhs].
 *
 * Return codes: 0 ok, 1 column out of range / above the diagonal,
 * 2 missing diagonal, 3 zero diagonal.
 */
#include <stdint.h>
#include <stddef.h>

/* Algorithm 1 (Section II), one right-hand side column at a time,
 * nonzeros visited in ascending column order. */
int oracle_forward_subst(int32_t n, const int32_t *row_ptr, const int32_t *col,
                         const double *val, const double *b, double *x,
                         int32_t nrhs)
{
    for (int32_t r = 0; r < nrhs; ++r) {
        for (int32_t i = 0; i < n; ++i) {
            double sum = b[(size_t)i * nrhs + r];
            double diag = 0.0;
            int have_diag = 0;
            for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                int32_t j = col[k];
                if (j < 0 || j > i) return 1;
                if (j == i) {
                    diag = val[k];
                    have_diag = 1;
                } else {
                    sum -= val[k] * x[(size_t)j * nrhs + r];
                }
            }
            if (!have_diag) return 2;
            if (diag == 0.0) return 3;
            x[(size_t)i * nrhs + r] = sum / diag;
        }
    }
    return 0;
}

/* Level of every row of DAG_L (Section II; level sets of Section II's
 * related work): 0 for a row with no off-diagonal entry, otherwise one more
 * than the deepest row it depends on.  Every stored off-diagonal entry is an
 * edge, whatever its value.  Returns the number of levels through *nlev. */
int oracle_levels(int32_t n, const int32_t *row_ptr, const int32_t *col,
                  int32_t *level, int32_t *nlev)
{
    int32_t deepest = -1;
    for (int32_t i = 0; i < n; ++i) {
        int32_t lv = 0;
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int32_t j = col[k];
            if (j < 0 || j > i) return 1;
            if (j < i && level[j] + 1 > lv) lv = level[j] + 1;
        }
        level[i] = lv;
        if (lv > deepest) deepest = lv;
    }
    *nlev = deepest + 1;
    return 0;
}

/* r = b - L x over every stored entry, diagonal included, row-major
 * [n][nrhs]; entries of a row summed in ascending column order. */
int oracle_spmv_lower(int32_t n, const int32_t *row_ptr, const int32_t *col,
                      const double *val, const double *b, const double *x,
                      double *r, int32_t nrhs)
{
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t c = 0; c < nrhs; ++c) {
            double s = b[(size_t)i * nrhs + c];
            for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                int32_t j = col[k];
                if (j < 0 || j > i) return 1;
                s -= val[k] * x[(size_t)j * nrhs + c];
            }
            r[(size_t)i * nrhs + c] = s;
        }
    }
    return 0;
}

/* Backward substitution over an upper-triangular CSR (every stored column
 * j >= i, diagonal stored): rows from n-1 down to 0, the row's off-diagonal
 * products subtracted in ascending column order, then the division by the
 * diagonal.  Same return codes, 1 meaning a column below the diagonal. */
int oracle_backward_subst(int32_t n, const int32_t *row_ptr, const int32_t *col,
                          const double *val, const double *b, double *x,
                          int32_t nrhs)
{
    for (int32_t r = 0; r < nrhs; ++r) {
        for (int32_t i = n - 1; i >= 0; --i) {
            double sum = b[(size_t)i * nrhs + r];
            double diag = 0.0;
            int have_diag = 0;
            for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                int32_t j = col[k];
                if (j < i || j >= n) return 1;
                if (j == i) {
                    diag = val[k];
                    have_diag = 1;
                } else {
                    sum -= val[k] * x[(size_t)j * nrhs + r];
                }
            }
            if (!have_diag) return 2;
            if (diag == 0.0) return 3;
            x[(size_t)i * nrhs + r] = sum / diag;
        }
    }
    return 0;
}
