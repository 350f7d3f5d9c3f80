// Triangular operators other than L x = b (sptrsv_analyze_ex).
//
// Every operator is brought to the lower-triangular form the rest of the
// library handles:
//   * U x = b (U upper): with P the exchange permutation (P x)_i = x_{n-1-i},
//     P U P is lower triangular and U x = b  <=>  (P U P)(P x) = P b.  Row i
//     of P U P is row n-1-i of U with columns c -> n-1-c, so the conversion
//     reverses the whole entry array (the mirror image of Sec. II's
//     forward substitution is the backward substitution).
//   * A^T x = b: the CSR of A^T (a stable sort of the entries by column), then
//     the rule above if A^T is upper.
// A solve structure built on P A P is translated back to A's numbering once
// (row ids, x columns, b columns), so the solve kernels read b and write x in
// the caller's order with no permuted copies.
#include "kernels.cuh"

namespace sptrsv {
namespace {

// row_ptr monotone inside [0, nnz] and every column in [0, n): checked
// before a transpose indexes arrays by column.  Same error word as
// validate_kernel (min of row << 8 | code).
__global__ void csr_check_kernel(int32_t n, int64_t nnz, const int32_t *__restrict__ row_ptr,
                                 const int32_t *__restrict__ col, unsigned long long *err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int code = 0;
    const int64_t a = row_ptr[i], e = row_ptr[i + 1];
    if ((i == 0 && a != 0) || a < 0 || e < a || e > nnz || (i == n - 1 && e != nnz)) {
        code = SPTRSV_ERR_UNSORTED;
    } else {
        for (int64_t k = a; k < e; ++k) {
            const int32_t c = col[k];
            if (c < 0 || c >= n) { code = SPTRSV_ERR_NOT_LOWER; break; }
        }
    }
    if (code) atomicMin(err, ((unsigned long long)i << 8) | (unsigned long long)code);
}

__global__ void reverse_ptr_kernel(int32_t n, int64_t nnz, const int32_t *__restrict__ rp,
                                   int32_t *__restrict__ orp) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    orp[i] = (int32_t)(nnz - rp[n - i]);
}

__global__ void reverse_entries_kernel(int32_t n, int64_t nnz, const int32_t *__restrict__ col,
                                       const double *__restrict__ val, int32_t *__restrict__ ocol,
                                       double *__restrict__ oval) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nnz) return;
    ocol[nnz - 1 - k] = n - 1 - col[k];
    oval[nnz - 1 - k] = val[k];
}

__global__ void entry_rows_kernel(int32_t n, const int32_t *__restrict__ rp,
                                  int32_t *__restrict__ rows) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) rows[k] = i;
}

__global__ void col_count_kernel(int64_t nnz, const int32_t *__restrict__ col, int32_t *cnt) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nnz) atomicAdd(&cnt[col[k]], 1);
}

__global__ void transpose_gather_kernel(int64_t nnz, const int32_t *__restrict__ order,
                                        const int32_t *__restrict__ rows,
                                        const double *__restrict__ val,
                                        int32_t *__restrict__ ocol, double *__restrict__ oval) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nnz) return;
    const int32_t e = order[k];
    ocol[k] = rows[e];
    oval[k] = val[e];
}

// Back to the caller's numbering: positions keep their place, the row a
// position solves and every x or b column are mirrored; pads and run slots
// (columns below -n) refer to positions and stay.
__global__ void struct_reverse_rows_kernel(int32_t n, int32_t *row_id) {
    const int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) row_id[p] = n - 1 - row_id[p];
}

__global__ void struct_reverse_cols_kernel(int32_t n, int64_t count, int32_t *ecol) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const int32_t c = ecol[k];
    if (c >= 0) ecol[k] = n - 1 - c;            // x term
    else if (c >= -n) ecol[k] = ~(n - 1 - ~c);  // b term ~j
}

// level[] by the caller's rows (a reversal) and perm[] in the caller's rows.
__global__ void levels_reverse_kernel(int32_t n, int32_t *level, int32_t *perm) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (level && i < n / 2) {
        const int32_t t = level[i];
        level[i] = level[n - 1 - i];
        level[n - 1 - i] = t;
    }
    if (perm) perm[i] = n - 1 - perm[i];
}

unsigned blocks_for(int64_t count, int threads) {
    return (unsigned)((count + threads - 1) / threads);
}

}  // namespace

cudaError_t launch_csr_check(int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col,
                             unsigned long long *err, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    csr_check_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, nnz, row_ptr, col, err);
    return cudaGetLastError();
}

cudaError_t launch_csr_reverse(int32_t n, int64_t nnz, const int32_t *rp, const int32_t *col,
                               const double *val, int32_t *orp, int32_t *ocol, double *oval,
                               cudaStream_t s) {
    reverse_ptr_kernel<<<blocks_for((int64_t)n + 1, 256), 256, 0, s>>>(n, nnz, rp, orp);
    if (nnz > 0)
        reverse_entries_kernel<<<blocks_for(nnz, 256), 256, 0, s>>>(n, nnz, col, val, ocol, oval);
    return cudaGetLastError();
}

cudaError_t launch_csr_transpose(int32_t n, int64_t nnz, const int32_t *rp, const int32_t *col,
                                 const double *val, int32_t *orp, int32_t *ocol, double *oval,
                                 int32_t *rows, int32_t *order, int32_t *cnt, int64_t *scan_tmp,
                                 void *radix_tmp, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)n * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    entry_rows_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, rp, rows);
    if (nnz > 0) col_count_kernel<<<blocks_for(nnz, 256), 256, 0, s>>>(nnz, col, cnt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = exclusive_scan_i32_i32(cnt, orp, n, scan_tmp, s)) != cudaSuccess) return e;
    if (nnz == 0) return cudaSuccess;
    // entries ordered by column; the sort is stable, so rows stay ascending
    // inside every column (= every row of A^T)
    if ((e = launch_level_perm((int32_t)nnz, col, n, order, radix_tmp, s)) != cudaSuccess) return e;
    transpose_gather_kernel<<<blocks_for(nnz, 256), 256, 0, s>>>(nnz, order, rows, val, ocol, oval);
    return cudaGetLastError();
}

cudaError_t launch_struct_reverse(int32_t n, int32_t *row_id, int64_t count, int32_t *ecol,
                                  cudaStream_t s) {
    if (n > 0) struct_reverse_rows_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, row_id);
    if (count > 0)
        struct_reverse_cols_kernel<<<blocks_for(count, 256), 256, 0, s>>>(n, count, ecol);
    return cudaGetLastError();
}

cudaError_t launch_levels_reverse(int32_t n, int32_t *level, int32_t *perm, cudaStream_t s) {
    if (n > 0) levels_reverse_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, level, perm);
    return cudaGetLastError();
}

}  // namespace sptrsv
