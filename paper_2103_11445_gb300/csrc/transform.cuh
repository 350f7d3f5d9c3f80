// Launchers of the rewriting and assembly kernels (transform.cu).
#pragma once

#include "kernels.cuh"

namespace sptrsv {

cudaError_t launch_expand_queries(int32_t nq, const int32_t *q_level, const int32_t *q_tgt,
                                  const int64_t *q_off, const int32_t *level_ptr,
                                  const int32_t *perm, int32_t *item_row, int32_t *item_tgt,
                                  int32_t *item_q, int32_t *item_pos, cudaStream_t s);
cudaError_t launch_rewrite_count(int64_t nitems, const int32_t *item_row,
                                 const int32_t *item_tgt, const int32_t *item_q,
                                 const int32_t *row_ptr, const int32_t *col,
                                 const int32_t *level, int cap, int32_t *fill_out,
                                 unsigned long long *added, int32_t *overflow,
                                 int32_t *maxlen, int num_sms, cudaStream_t s);
// acc[l][11] (zeroed): rows, off-diagonal entries, 8 log2 length bins and
// the ancestor span of level l (the per-level analysis features)
cudaError_t launch_level_counts(int32_t n, const int32_t *row_ptr, const int32_t *col,
                                const int32_t *level, unsigned long long *acc, cudaStream_t s);
// out[level] = most off-diagonal terms of a row of that level (out zeroed)
cudaError_t launch_level_max(int32_t n, const int32_t *level, const int32_t *offdeg, int32_t *out,
                             cudaStream_t s);
// finish[row] = hop + terms(row) + max finish of its dependencies, for the
// rows of chunks [c0, c1) (one level of a solve structure; chunk_run_p0 may
// be null when no entry encodes a run slot)
cudaError_t launch_critpath_level(int32_t c0, int32_t c1, int L, int32_t n, const int4 *meta,
                                  const int32_t *ecol, const int32_t *row_id,
                                  const int32_t *chunk_run_p0, int64_t hop, int64_t *finish,
                                  cudaStream_t s);
cudaError_t launch_rewrite_numeric(int64_t nitems, const int32_t *item_row,
                                   const int32_t *item_tgt, const int64_t *out_off,
                                   const int32_t *row_ptr, const int32_t *col,
                                   const double *val, const int32_t *level, int cap,
                                   int32_t *out_col, double *out_val, int32_t *nb_out,
                                   DevStatus *st, int num_sms, cudaStream_t s);
cudaError_t launch_pos_item(int32_t n, int64_t nitems, const int32_t *item_pos,
                            int32_t *pos_item, cudaStream_t s);
cudaError_t launch_chunk_width(int32_t nchunks, const int32_t *c_row0, const int32_t *c_nrows,
                               int L, const int32_t *perm, const int32_t *offdeg,
                               const int32_t *pos_item, const int64_t *rw_off, int64_t *slots,
                               int32_t *width, cudaStream_t s);
template <typename T>
cudaError_t launch_chunk_fill(int32_t nchunks, int L, const int32_t *c_row0,
                              const int32_t *c_nrows, const int32_t *c_width,
                              const int64_t *c_off, const int32_t *perm, const int32_t *row_ptr,
                              const int32_t *col, const double *val, const int32_t *pos_item,
                              const int64_t *rw_off, const int32_t *rw_col,
                              const double *rw_val, int4 *meta, int32_t *ecol, T *eval,
                              int32_t *row_id, T *diag, cudaStream_t s);
// Export (tests): x terms (including run slots, decoded back to rows) and b
// terms per original row.
cudaError_t launch_export_count(int32_t nchunks, int L, const int4 *meta, const int32_t *ecol,
                                const int32_t *row_id, int32_t n, int64_t *xcnt, int64_t *bcnt,
                                cudaStream_t s);
cudaError_t launch_export_fill(int32_t nchunks, int L, const int4 *meta, const int32_t *ecol,
                               const double *eval, const int32_t *row_id,
                               const int32_t *chunk_level, const int32_t *chunk_run_p0,
                               int32_t n, const int64_t *xptr, const int64_t *bptr,
                               int32_t *xcol, double *xval, int32_t *bcol, double *bw,
                               int32_t *new_level, cudaStream_t s);
cudaError_t launch_chunk_level(int32_t nlev, const int32_t *lvl_chunk, int32_t *chunk_level,
                               cudaStream_t s);
cudaError_t launch_f64_to_f32(const double *a, float *b, int64_t n, cudaStream_t s);
// Encodes the x terms of run chunks that read a row of their own run as
// shared-memory slots (see SolveData::run_slots).  pos_tmp: int32[n].
cudaError_t launch_encode_runs(int32_t n, int L, const int32_t *row_id, const int4 *meta,
                               int32_t nrc, const int32_t *run_chunk, const int2 *run_span,
                               int32_t *pos_tmp, int32_t *ecol, cudaStream_t s);

// Single-CTA tail segments (tail.cuh TailData): pos[row_id[i]] = i; per
// segment row the counts of folded and in-segment terms (chunks
// c0..nchunks-1, rows numbered from solve position P0), the largest
// in-segment count in *kmax, *bad = 1 if an entry is a run slot; then the
// records (terms packed as (slot or column, 0, value bits), coefficients
// divided by the diagonal unless a row is marked kTailUnscaled).
cudaError_t launch_pos_of_row(int32_t n, const int32_t *row_id, int32_t *pos, cudaStream_t s);
cudaError_t launch_tail_count(int32_t c0, int32_t nchunks, int L, int32_t n, const int4 *meta,
                              const int32_t *ecol, const int32_t *pos_of, int32_t P0,
                              int32_t *cnt_a, int32_t *cnt_n, int32_t *kmax, int32_t *bad,
                              cudaStream_t s);
cudaError_t launch_tail_fill(int32_t c0, int32_t nchunks, int L, int32_t n, const int4 *meta,
                             const int32_t *ecol, const double *eval, const int32_t *row_id,
                             const double *diag, const int32_t *chunk_level, int32_t lev0,
                             const int32_t *tlp, const int32_t *pos_of, int32_t P0, int32_t W,
                             int32_t T, int32_t K, int32_t nr, const int64_t *aptr,
                             int32_t *trow, double2 *tdiag, int32_t *tnn, int4 *term,
                             int32_t *acol, double *aval, cudaStream_t s);

}  // namespace sptrsv
