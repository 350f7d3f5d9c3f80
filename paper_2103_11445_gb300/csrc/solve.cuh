// Solve kernels (solve.cu): structure of the level-ordered solve data and the
// launchers.
#pragma once

#include "kernels.cuh"

namespace sptrsv {

// Level-ordered solve structure (device pointers).  Rows are stored in solve
// order (level by level); each level is cut into chunks of H = 32 / L rows.
// Chunk c: meta[c] = (first solve position, rows, width, entry offset).
// Entry j of row k of the chunk sits at
//     off + (j / L) * (rows * L) + k * L + (j % L)
// so the chunk's active lanes read consecutive words every step.  ecol >= 0
// is an x term, ecol < 0 (not PAD_COL) a b term of a rewritten row.
template <typename T>
struct SolveData {
    int32_t n;                  // rows
    int32_t nlev;
    int32_t nchunks;
    int32_t L;                  // lanes per row of the layout
    const int32_t *lvl_chunk;   // [nlev + 1]
    const int4 *meta;           // [nchunks]
    const int32_t *ecol;
    const T *eval;
    const int32_t *row_id;      // solve position -> row
    const T *diag;              // solve position p -> (L_ii, RN(1/L_ii) or 0) at [2p], [2p+1]
    const int2 *phases;         // barrier schedule: (l0, l1) level, or (l0, -l1) CTA-local run
    int32_t nphases;
    int32_t backoff_ns;         // sleep between failed polls (synchronisation-free), 0 = none
    // CTA-local runs keep the unknowns they produce in shared memory: entries
    // of run chunks that read a row of the same run are encoded as
    // col = -(n + 1) - slot, slot = solve position - first position of the
    // run; run_slots = largest run (rows), 0 when there are no runs.
    int32_t run_slots;
    // Staging of the synchronisation-free solve (one right-hand side): chunks
    // of at most stage_z steps per lane are copied into shared memory by the
    // bulk-copy engine one chunk ahead; 0 = no staging.  row_id must hold 4
    // spare elements past n and diag 8 (aligned over-reads of the copies).
    int32_t stage_z;
    // Chunk schedule of the synchronisation-free kernels for a grid of
    // sched_nw warps: warp w solves sched[sched_ptr[w] .. sched_ptr[w + 1])
    // in that order (level by level, the level's chunks dealt out to warps
    // 0, 1, ... in turn).  Null, or another warp count: chunk c goes to warp
    // c mod (warps), in chunk order.
    const int32_t *sched;
    const int32_t *sched_ptr;
    int32_t sched_nw;
    // Chunk blobs of the staged kernels (BlobLayout): chunk c occupies the
    // 16-byte units [bofs[c], bofs[c + 1]) of blob.
    const uint4 *blob;
    const int64_t *bofs;
    // Level-timed solve (staged kernel only): level_ns[0] = the start of the
    // solve, level_ns[1 + g] = the latest completion time of a chunk of new
    // level g (%globaltimer); null: no stamps.  chunk_level[c] = new level
    // of chunk c.
    const int32_t *chunk_level;
    unsigned long long *level_ns;
};

// One chunk as one contiguous run of 16-byte units: unit 0 the chunk
// descriptor (first position, rows y, steps z, entry offset), then the row
// ids (y int32), the diagonal pairs (2y elements), the columns (z y L int32,
// in the entry order of ecol) and the values (z y L elements), each padded
// to whole units.
template <typename T>
struct BlobLayout {
    int rows, diag, cols, vals, units;   // unit offsets, total units
    __host__ __device__ BlobLayout(int y, int z, int L) {
        const int ne = z * y * L;
        rows = 1;
        diag = rows + (4 * y + 15) / 16;
        cols = diag + (2 * y * (int)sizeof(T) + 15) / 16;
        vals = cols + (4 * ne + 15) / 16;
        units = vals + ((int)sizeof(T) * ne + 15) / 16;
    }
};

// Builds the blobs of a structure: bofs[nchunks + 1] (exclusive prefix of
// the chunks' units, computed here) and blob (units: bofs[nchunks]); the
// caller allocates blob after reading the total (two phases).
template <typename T>
cudaError_t launch_blob_units(int32_t nchunks, int L, const int4 *meta, int64_t *units,
                              cudaStream_t s);
template <typename T>
cudaError_t launch_blob_fill(int32_t nchunks, int L, const int4 *meta, const int32_t *row_id,
                             const T *diag, const int32_t *ecol, const T *eval,
                             const int64_t *bofs, uint4 *blob, cudaStream_t s);

// Largest staging width (steps per lane) the kernels accept (at most 32: a
// lane notes its late steps in one 32-bit mask).
constexpr int kStageZMax = 24;
// Resident warps per SM whose slots the default staging width must fit.
constexpr int kStageWarpsPerSM = 16;
// Largest staging width whose slots, for `warps` resident warps of the
// layout with L lanes per row, fit in `smem_per_sm` bytes of shared memory
// (with 1 KiB per CTA reserved).
template <typename T>
int stage_cap_z(int L, int smem_per_sm, int warps);

struct LaunchCfg {
    int block_threads;   // threads per CTA
    int grid;            // CTAs (co-resident)
};

// x = L^{-1} rhs for `nr` right-hand sides stored with leading dimension ld
// (row i, column r at [i * ld + r]).  rhs is FP64; out has type T.
// syncfree selects the synchronisation-free kernel (it pre-fills out with
// the "not computed" sentinel itself, then one grid barrier).  `skip_if_converged`: the kernels return
// at once when st->ir_flag is set (refinement loop).
template <typename T>
cudaError_t launch_solve(const SolveData<T> &sd, const double *rhs, T *out, int32_t n,
                         int ld, int nr, bool syncfree, const LaunchCfg &cfg,
                         DevStatus *st, uint64_t timeout_ns, bool skip_if_converged,
                         cudaStream_t s);

// Largest co-resident grid for the chosen kernel (CTAs per SM * SMs), with
// the dynamic shared memory the barrier kernel's runs need.
template <typename T>
int max_coresident_ctas(int L, int nr, bool syncfree, int block_threads, int num_sms,
                        int run_slots = 0, int stage_z = 0);

// ---------------------------------------------------------------------------
// Batched solve: many independent plans in one persistent launch.  Matrix m
// owns CTAs [cta_begin, cta_begin + cta_count); all CTAs are co-resident, a
// group solves its matrix synchronisation-free and separates the phases of
// the refinement with a barrier on its own counter (never a grid barrier).
constexpr int kBatchMaxIter = 16;

struct BatchMat {
    SolveData<float> s32;     // FP32 structure (refinement)
    SolveData<double> s64;    // FP64 structure (direct solve)
    const int32_t *row_ptr;   // the analysed lower triangle, for the FP64 residual
    const int32_t *col;
    const double *val;
    int32_t rev;              // the CSR is P A P (see residual_kernel)
    const double *b;          // [n, nr] row-major
    double *x;
    float *d32;               // scratch [n, nr]
    double *r64;              // scratch [n, nr]
    double lnorm;             // |L|_inf
    int32_t n, nr, R;         // rows, right-hand sides, lanes per row group (pow2 >= nr)
    int32_t cta_begin, cta_count;
};

struct BatchCtl {             // per matrix, zeroed before every launch
    unsigned long long bar;
    unsigned long long norms[kBatchMaxIter + 1][3];  // |r|, |x| per check; [0][2] = |b|
    int32_t iters;            // corrections applied
    int32_t converged;
    unsigned long long t_begin, t_end;  // %globaltimer: first CTA in, last CTA out
};

// ir: FP32 solves + FP64 refinement (plans in SPTRSV_F32_IR precision);
// otherwise one FP64 solve per matrix.
cudaError_t launch_batch(const BatchMat *mats, int32_t nmats, BatchCtl *ctl, DevStatus *st,
                         bool ir, double tol, int max_iter, uint64_t timeout_ns, int block_threads,
                         int grid, cudaStream_t s);
int batch_max_coresident(bool ir, int block_threads, int num_sms);

// FP64 residual r = b - L x over the original CSR, with infinity norms of r
// and x accumulated in st->norms[0], [1]; returns at once when ir_flag is set.
// r = b - A x; rev: the CSR holds P A P (see residual_kernel).
cudaError_t launch_residual(int32_t n, const int32_t *row_ptr, const int32_t *col,
                            const double *val, bool rev, const double *b, const double *x,
                            double *r, int nr, int ld, DevStatus *st, cudaStream_t s);
// Refinement bookkeeping.
cudaError_t launch_ir_begin(DevStatus *st, const double *b, int64_t count, cudaStream_t s);
cudaError_t launch_ir_decide(DevStatus *st, double tol, const unsigned long long *lnorm,
                             cudaStream_t s);
// x = (double) d (first step), or x += d (later steps, skipped when converged)
cudaError_t launch_ir_update(double *x, const float *d, int64_t count, bool first,
                             DevStatus *st, cudaStream_t s);

}  // namespace sptrsv
