// Single-CTA tail of the solve (tail.cu): structure and launcher.
#pragma once

#include "kernels.cuh"

namespace sptrsv {

// One segment of the single-CTA tail: a run of trailing levels (each at most
// blockDim rows) solved by one CTA after everything before it.  Segment rows
// are numbered by solve position relative to the segment's first one.
//   lp[nlev + 1]        level starts (relative positions)
//   row, diag           per row: its row index, (L_ii, RN(1/L_ii) or 0)
//   nn                  per row: in-segment term count (bits 0-7), mask of
//                       the terms read from x (bits 8-23), kTailUnscaled
//   term [K][nrows]     in-segment terms (x, 0, value bits): x a shared-
//                       memory slot (position mod W), or for a term in the
//                       mask the row x is read from; unused: (0, 0, 0.0)
//   aptr, acol, aval    the other terms (acol >= 0: an unknown solved before
//                       the segment, acol < 0: b[~acol]), folded into s0
// Coefficients (term values, aval) are divided by the row's diagonal unless
// the row is marked kTailUnscaled.
struct TailData {
    int32_t nrows, nlev, K, W;
    const int32_t *lp, *row, *nn;
    const int4 *term;
    const double2 *diag;
    const int64_t *aptr;
    const int32_t *acol;
    const double *aval;
    double *s0;
};
// s0 = b_row / L_ii - (other terms) (b_row - ... for an unscaled row), then
// the segment; one right-hand side, FP64.
cudaError_t launch_tail(const TailData &td, const double *b, double *x, int block_threads,
                        cudaStream_t s);
// The fold pass alone (s0 of every segment row).
cudaError_t launch_tail_fold(const TailData &td, const double *b, const double *x,
                             cudaStream_t s);

}  // namespace sptrsv
