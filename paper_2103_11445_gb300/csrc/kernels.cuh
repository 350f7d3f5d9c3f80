// Host-side launchers of the library's kernels (one group per .cu file).
// All launchers are stream-ordered and return the cudaError_t of the launch.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace sptrsv {

// ---- scan.cu --------------------------------------------------------------
// out[0..n] = exclusive prefix sums of in[0..n), out[n] = total.
// `tmp` must hold scan_tmp_elems(n) int64 values.
int64_t scan_tmp_elems(int64_t n);
cudaError_t exclusive_scan_i32_i64(const int32_t *in, int64_t *out, int64_t n,
                                   int64_t *tmp, cudaStream_t s);
cudaError_t exclusive_scan_i64_i64(const int64_t *in, int64_t *out, int64_t n,
                                   int64_t *tmp, cudaStream_t s);
cudaError_t exclusive_scan_i32_i32(const int32_t *in, int32_t *out, int64_t n,
                                   int64_t *tmp, cudaStream_t s);

// ---- analyze.cu -----------------------------------------------------------
// Validation: err (u64, host-initialised to ~0) receives min(row<<8 | code)
// over bad rows; offdeg[i] = off-diagonal count; lnorm (u64 bits) = max row
// abs sum.
cudaError_t launch_validate(int32_t n, int64_t nnz, const int32_t *row_ptr,
                            const int32_t *col, const double *val,
                            int32_t *offdeg, unsigned long long *err,
                            unsigned long long *lnorm, cudaStream_t s);
// Level analysis by a synchronisation-free pass in row order (one
// cooperative launch, no barrier per level): level[i] for every row,
// *nlev_out = 1 + deepest level.  level and nlev_out are initialised here.
cudaError_t launch_levels_syncfree(int32_t n, const int32_t *row_ptr, const int32_t *col,
                                   int32_t *level, int32_t *nlev_out, DevStatus *st,
                                   uint64_t timeout_ns, int num_sms, cudaStream_t s);
// level_ptr[0..nlev] from the level-ordered permutation.
cudaError_t launch_level_ptr(int32_t n, const int32_t *level, const int32_t *perm, int32_t nlev,
                             int32_t *level_ptr, cudaStream_t s);
// histogram of rows by off-diagonal count (bins 0 | 1-2 | 3-6 | >= 7)
cudaError_t launch_offdeg_hist(int32_t n, const int32_t *offdeg, unsigned long long *bins,
                               cudaStream_t s);
// perm = rows ordered by (level, row), via a stable LSD radix sort.
// tmp must hold radix_tmp_bytes(n) bytes.
size_t radix_tmp_bytes(int32_t n);
cudaError_t launch_level_perm(int32_t n, const int32_t *level, int32_t nlev,
                              int32_t *perm, void *tmp, cudaStream_t s);

// ---- operator.cu ----------------------------------------------------------
// Structural check before a transpose: row_ptr monotone inside [0, nnz],
// columns in [0, n).  err as for launch_validate.
cudaError_t launch_csr_check(int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col,
                             unsigned long long *err, cudaStream_t s);
// B = P A P, P the exchange permutation (turns an upper triangle into a lower
// one and back).
cudaError_t launch_csr_reverse(int32_t n, int64_t nnz, const int32_t *rp, const int32_t *col,
                               const double *val, int32_t *orp, int32_t *ocol, double *oval,
                               cudaStream_t s);
// B = A^T with ascending columns in every row.  Scratch: rows[nnz],
// order[nnz], cnt[n], scan_tmp[scan_tmp_elems(n)], radix_tmp of
// radix_tmp_bytes(nnz) bytes.
cudaError_t launch_csr_transpose(int32_t n, int64_t nnz, const int32_t *rp, const int32_t *col,
                                 const double *val, int32_t *orp, int32_t *ocol, double *oval,
                                 int32_t *rows, int32_t *order, int32_t *cnt, int64_t *scan_tmp,
                                 void *radix_tmp, cudaStream_t s);
// Solve structure built on P A P -> the caller's numbering (row ids, x and b
// columns mirrored; pads and run slots kept).
cudaError_t launch_struct_reverse(int32_t n, int32_t *row_id, int64_t count, int32_t *ecol,
                                  cudaStream_t s);
// Level export of a mirrored plan in the caller's rows: level[] reversed,
// perm[] entries mirrored (either may be null).
cudaError_t launch_levels_reverse(int32_t n, int32_t *level, int32_t *perm, cudaStream_t s);

}  // namespace sptrsv
