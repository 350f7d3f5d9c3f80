// Single-CTA tail of the solve (tail.cu): structure and launcher.
#pragma once

#include "kernels.cuh"

namespace sptrsv {

// Single-CTA tail: the trailing levels (each at most blockDim rows) solved by
// one CTA after the main kernel has solved the levels before them.  Tail
// rows are numbered by solve position relative to the tail's first one.
//   lp[nlev + 1]        level starts (relative positions)
//   row, diag, nn       per row: its row index, (L_ii, RN(1/L_ii) or 0), the
//                       number of in-tail terms
//   tcol, tval [K][nrows]  in-tail terms: tcol >= 0 a shared-memory slot
//                       (position mod W), tcol < 0 the row ~tcol read from x;
//                       unused slots hold (0, 0.0)
//   aptr, acol, aval    the other terms (acol >= 0: an unknown solved before
//                       the tail, acol < 0: b[~acol]), folded into s0
struct TailData {
    int32_t nrows, nlev, K, W;
    const int32_t *lp, *row, *nn, *tcol;
    const double2 *diag;
    const double *tval;
    const int64_t *aptr;
    const int32_t *acol;
    const double *aval;
    double *s0;
};
// s0 = b_row - (other terms), then the tail; one right-hand side, FP64.
cudaError_t launch_tail(const TailData &td, const double *b, double *x, int block_threads,
                        cudaStream_t s);

}  // namespace sptrsv
