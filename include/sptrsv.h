/*
 * sptrsv.h -- C ABI of the GB300 sparse lower-triangular solver with
 * equation rewriting (Yilmaz, "Graph Transformation and Specialized Code
 * Generation for Sparse Triangular Solve (SpTRSV)", arXiv:2103.11445).
 *
 * The problem (Sec. II): solve L x = b for a sparse lower-triangular L stored
 * in CSR (Fig. 1).  Rows are grouped into levels of the dependency graph
 * DAG_L; levels run one after another.  Sec. III rewrites the equations of
 * rows in thin levels by substituting the equations of their dependencies,
 * which lifts those rows into earlier levels and removes levels (and the
 * synchronisation at their ends).  Rearranged back into L x = b form
 * (Fig. 3) a rewritten row keeps its diagonal, depends on fewer and earlier
 * unknowns, and carries a right-hand side  b_i - sum_j c_j b_j.
 *
 * Conventions that hold for every call:
 *  - Pointers prefixed d_ are device pointers of the current CUDA device,
 *    h_ are host pointers.  All caller buffers stay owned by the caller; the
 *    library never frees them and keeps no reference after a call returns.
 *  - CSR: row_ptr int32[n+1] (row_ptr[0] == 0, non-decreasing), col
 *    int32[nnz] strictly ascending inside each row, every column <= its row,
 *    the diagonal stored (as the last entry of the row) and non-zero.
 *    Values are FP64.  Every stored off-diagonal entry is a dependency, even
 *    an explicit 0.0.
 *  - Right-hand sides and solutions are row-major [n][nrhs], contiguous
 *    (the layout of a C-contiguous torch tensor of shape (n, nrhs)).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  sptrsv_solve and sptrsv_batch_solve are asynchronous with
 *    respect to the host; sptrsv_analyze and sptrsv_transform synchronise
 *    the stream because the host needs level counts to plan.
 *  - Errors the host can see are returned at once.  Errors a kernel finds
 *    (invalid CSR, a bounded wait that ran out) are latched in the plan and
 *    returned by the next sptrsv_check (which synchronises) or by the next
 *    synchronising call.  A plan with a latched error refuses further work
 *    with SPTRSV_ERR_BAD_STATE until it is destroyed.
 *  - A plan is used by one host thread at a time; solves on one plan must not
 *    overlap on the device (they share the plan's scratch).
 */
#ifndef SPTRSV_H
#define SPTRSV_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SPTRSV_API __attribute__((visibility("default")))
#else
#define SPTRSV_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPTRSV_OK = 0,
    SPTRSV_ERR_INVALID_ARG = 1,   /* null pointer, negative size, x aliases b */
    SPTRSV_ERR_NOT_LOWER = 2,     /* a column above the diagonal or out of range */
    SPTRSV_ERR_UNSORTED = 3,      /* columns of a row not strictly ascending,
                                     or row_ptr not non-decreasing */
    SPTRSV_ERR_ZERO_DIAG = 4,
    SPTRSV_ERR_MISSING_DIAG = 5,
    SPTRSV_ERR_OOM = 6,           /* device allocation failed */
    SPTRSV_ERR_CUDA = 7,          /* a CUDA runtime call failed */
    SPTRSV_ERR_TIMEOUT = 8,       /* a bounded device wait gave up */
    SPTRSV_ERR_BAD_STATE = 9,     /* call out of order or plan already failed */
    SPTRSV_ERR_UNSUPPORTED = 10,  /* size or mode the library does not handle */
    SPTRSV_ERR_BREAKDOWN = 11,    /* an iteration met a non-finite residual or a
                                     non-positive curvature (p, A p) */
    SPTRSV_ERR_CODEGEN = 12       /* generated code requested but the runtime
                                     compiler is missing or rejected it */
} sptrsv_status_t;

typedef struct sptrsv_plan_s *sptrsv_plan_t;    /* opaque, owned by the library */
typedef struct sptrsv_batch_s *sptrsv_batch_t;  /* opaque, owned by the library */
typedef struct sptrsv_mlp_s *sptrsv_mlp_t;      /* opaque, owned by the library */
typedef struct sptrsv_pcg_s *sptrsv_pcg_t;      /* opaque, owned by the library */
typedef void *sptrsv_stream_t;                  /* cudaStream_t */

/* Row selection for the rewriting (Sec. III; the paper chooses rows by
 * hand, Sec. IV). */
enum {
    SPTRSV_SELECT_NONE = 0,       /* plain level sets, nothing rewritten */
    SPTRSV_SELECT_HEURISTIC = 1,  /* thin-level heuristic H (below) */
    SPTRSV_SELECT_COSTMODEL = 2,  /* learned cost model picks the rewrite
                                     (sptrsv_set_costmodel or
                                     sptrsv_costmodel_load; else H) */
    SPTRSV_SELECT_FIXED = 3,      /* merge every `depth`+1 consecutive levels */
    SPTRSV_SELECT_AUTO = 4,       /* measured: times the candidates below on
                                     the plan and keeps the fastest */
    SPTRSV_SELECT_CRITPATH = 5,   /* minimises the critical path of the
                                     synchronisation-free solve (below) */
    SPTRSV_SELECT_SEGMODEL = 6    /* per-segment learned cost: a network
                                     predicts the time each candidate segment
                                     adds, depths chosen per segment (below;
                                     without a network: SELECT_CRITPATH) */
};
/* SPTRSV_SELECT_SEGMODEL (the matrix-analysis module deciding which levels
 * to rewrite and how deep, Sec. IV): for every kept level t and depth
 * d <= min(max_depth, 4) (the depths of its training data) the segment's
 * features (sptrsv_segment_features)
 * go through the process-wide segment network (sptrsv_segmodel_load), whose
 * output is the log2 of the time in microseconds the segment's new level
 * adds to the solve; the segmentation minimising the sum of those times is
 * found by dynamic programming over the levels, as for SELECT_CRITPATH. */
/* SPTRSV_SELECT_CRITPATH (the rewriting applied to synchronisation-free
 * execution, Sec. III): a row finishes one hop after the latest of its
 * dependencies plus its own terms, f(i) = hop_weight + terms(i) + max f(dep).
 * If every row of a new level waits for the whole level before it, the
 * plan's critical path is the sum over new levels of hop_weight + (most
 * terms of a row in it) -- an upper bound of the weighted critical path of
 * the transformed system.  The segmentation minimising that sum is found by
 * dynamic programming over the levels (last level first, ties to the
 * smaller depth), each segment absorbing at most max_depth levels with no
 * rewritten row above max_row_fill terms; every lift (level l rewritten to
 * l - r, r <= max_depth) is counted on the device first, so the cost grows
 * with max_depth. */
/* SPTRSV_SELECT_AUTO: the candidates are the plain level sets (code 0),
 * merging every d+1 levels for d = 1, 2, 3 (code d), heuristic H with the
 * given thin_rows / max_depth / flop_budget (code 200), H on the levels of
 * fewer than 32 rows, up to 8 or 16 deep, within 4x the plain FLOPs (codes
 * 108, 116), the critical-path selection with at most 4 levels per segment
 * (code 300), and the cost model's pick when a network is available (its
 * code).  Each is built and timed with the synchronisation-free kernel at 1
 * and at 4 lanes per row (one warm-up and three solves of a vector of ones,
 * the fastest counts); the fastest candidate is then transformed with the
 * caller's solve_mode (SOLVE_AUTO: launch autotuning as usual).
 * sptrsv_info_t.chosen_depth is its code; transform_ms covers the search. */
/* Solve kernels.  BARRIER: persistent grid, one grid barrier per level (or
 * per run of thin levels kept inside one CTA).  SYNCFREE: no barriers, each
 * row waits for the unknowns it reads (Sec. II).  AUTO: the autotuner times
 * both on the plan. */
enum { SPTRSV_SOLVE_AUTO = 0, SPTRSV_SOLVE_BARRIER = 1, SPTRSV_SOLVE_SYNCFREE = 2 };
enum { SPTRSV_F64 = 0, SPTRSV_F32_IR = 1 };

/* Parameters of sptrsv_transform.  Fill with sptrsv_default_params first.
 *
 * Heuristic H: levels are scanned in order; each new level starts at a kept
 * level t and absorbs the following levels t+1, t+2, ... (their rows are
 * rewritten to depend only on levels < t) while the next level has fewer
 * than `thin_rows` rows, at most `max_depth` levels have been absorbed, no
 * rewritten row would exceed `max_row_fill` off-diagonal terms, and the FLOPs
 * added over the whole matrix stay <= flop_budget * FLOPs of the plain solve
 * (FLOPs: 2 per off-diagonal term, x or b, plus 1 per row). */
typedef struct {
    int32_t select_mode;     /* SPTRSV_SELECT_* (default HEURISTIC) */
    int32_t depth;           /* FIXED mode: levels absorbed per new level */
    int32_t thin_rows;       /* tau; <= 0: number of resident warps / 4 */
    int32_t max_depth;       /* d_max, 0..16 (default 8) */
    double flop_budget;      /* rho; < 0: 0.10 (the +10% of Sec. V) */
    int32_t max_row_fill;    /* cap on off-diagonal terms of a rewritten row
                                (default 1024, at most 4096) */
    int32_t solve_mode;      /* SPTRSV_SOLVE_* (default AUTO = autotune) */
    int32_t precision;       /* SPTRSV_F64 or SPTRSV_F32_IR */
    double ir_tol;           /* F32_IR: stop when |b - L x|_inf <=
                                ir_tol * (|L|_inf |x|_inf + |b|_inf); default 1e-15 */
    int32_t ir_max_iter;     /* F32_IR: refinement steps at most (default 8,
                                0 = plain FP32 solve, < 0 = default, max 64) */
    int32_t lanes_per_row;   /* 1,2,4,8,16,32; 0 = auto */
    int32_t block_threads;   /* 64..512, multiple of 32; 0 = auto */
    int32_t cta_run_rows;    /* levels of at most this many rows run inside
                                one CTA (no grid barrier); 0 = auto, <0 = off */
    int32_t wait_timeout_ms; /* bound on every device wait (default 5000); a
                                solve longer than this is reported as TIMEOUT */
    int32_t grid_blocks;     /* CTAs of the persistent solve (clipped to the
                                co-resident maximum); 0 = auto */
    int32_t poll_backoff_ns; /* synchronisation-free solve: sleep between
                                polls of an unready unknown; 0 = none,
                                < 0 = auto */
    int32_t nrhs_hint;       /* right-hand sides a solve usually carries
                                (1..32; default 1).  Above 1 the structure is
                                laid out for that many columns (one warp lane
                                per column and row, a chunk's rows in one
                                pass) and the autotuner times solves with
                                that many columns; any nrhs still works. */
    int32_t tail_rows;       /* single-CTA tail: the longest run of trailing
                                levels with at most this many rows each (at
                                least 8 levels, <= 256 rows) is solved by one
                                CTA after the main kernel, with the unknowns
                                it produces kept in shared memory and the
                                terms from before it folded into one constant
                                per row by a grid-wide pre-pass.  Used for
                                one right-hand side in FP64.  0 = auto
                                (SOLVE_AUTO times 32, 64, 128 and 256 rows and
                                keeps the tail only if faster; none
                                otherwise), < 0 = never, > 256 = 256. */
    int32_t stage_z;         /* synchronisation-free solve of one right-hand
                                side: each warp's next chunks of rows (row
                                ids, diagonals, columns, values divided by
                                the diagonal) are copied into shared memory
                                by asynchronous copies while the warp solves
                                the current one, for chunks that fit a slot
                                sized for stage_z steps per lane; larger
                                chunks read global memory.  0 = auto (the
                                width of 99% of the chunks, capped so that
                                the slots of 16 resident warps fit an SM's
                                shared memory), < 0 = off, > 24 = 24. */
    int32_t hop_weight;      /* SELECT_CRITPATH: weight of one dependency hop
                                in units of one term of a row (<= 0: 16) */
    int32_t codegen_rows;    /* per-matrix generated code (the GPU form of the
                                paper's specialised code generation, Sec. IV):
                                a segment of the single-CTA tail (tail_rows >
                                0) with at most codegen_rows rows and fewer
                                than 16 terms per level on average is solved
                                by a kernel generated for it, its row ids,
                                unknown slots and coefficients written into
                                the code as constants, compiled at transform
                                time by the runtime compiler (NVRTC) and run
                                by one thread in solve order, without
                                barriers (thin segments: chains, two-row
                                levels).  0 = off (default); at most 4096
                                (compiling takes about 1.3 ms per row). */
} sptrsv_transform_params_t;

/* Everything a caller may want to report about a plan. */
typedef struct {
    int32_t n;
    int64_t nnz;
    int32_t nlev;            /* levels of DAG_L */
    int32_t nlev_new;        /* levels solved after the transform */
    int32_t rows_rewritten;
    int64_t nnz_x;           /* off-diagonal x terms in the solve structure */
    int64_t nnz_b;           /* b terms of rewritten rows */
    int64_t flops_plain;     /* per right-hand side: 2 (nnz - n) + n */
    int64_t flops_new;       /* 2 (nnz_x + nnz_b) + n */
    int32_t select_mode, solve_mode, precision;
    int32_t lanes_per_row, block_threads, grid_blocks, cta_run_rows;
    int32_t thin_rows, max_depth;
    double flop_budget;
    int32_t ir_iters_last;   /* refinement steps of the last F32_IR solve
                                (valid after a synchronisation) */
    int32_t num_sms;
    int32_t poll_backoff_ns;
    int32_t chosen_depth;    /* SELECT_COSTMODEL: candidate code the network picked
                                (-1 when it did not run) */
    double analyze_ms, transform_ms;
    int32_t op;              /* SPTRSV_OP_* of the plan */
    int32_t tuned_from_cache; /* 1: the last SOLVE_AUTO transform reused the launch
                                 tuned earlier in this process for a plan of the
                                 same shape (sptrsv_autotune_cache_clear) */
    int32_t tail_rows;       /* width limit of the single-CTA tail in use (0: none) */
    int32_t tail_levels;     /* levels it solves */
    int32_t stage_z;         /* staging width of the FP64 one-column solve in
                                use (0: not staged) */
    int32_t codegen_segments; /* tail segments solved by generated kernels */
    double codegen_ms;       /* time the last transform spent generating and
                                compiling them */
} sptrsv_info_t;

SPTRSV_API const char *sptrsv_status_string(sptrsv_status_t s);
SPTRSV_API void sptrsv_default_params(sptrsv_transform_params_t *prm);

/* Level analysis of DAG_L (Sec. II; level sets as in Sec. II's related
 * work, built here on the device by validation and a synchronisation-free
 * pass over the rows in order -- each row's level is one more than the
 * deepest of its dependencies -- then a stable sort of the rows by level;
 * Sec. IV's matrix-analysis module).
 * Copies the CSR into the plan, so the caller may free it afterwards.
 * Returns the validation error codes above for malformed CSR.  On success
 * *out is a plan that solves the plain level sets. */
SPTRSV_API sptrsv_status_t sptrsv_analyze(int32_t n, int64_t nnz, const int32_t *d_row_ptr,
                               const int32_t *d_col, const double *d_val,
                               sptrsv_stream_t stream, sptrsv_plan_t *out);

/* Which triangular system a plan solves, given the CSR of A. */
typedef enum {
    SPTRSV_OP_LOWER = 0,        /* A lower triangular: A x = b (sptrsv_analyze) */
    SPTRSV_OP_UPPER = 1,        /* A upper triangular: A x = b */
    SPTRSV_OP_LOWER_TRANS = 2,  /* A lower triangular: A^T x = b */
    SPTRSV_OP_UPPER_TRANS = 3   /* A upper triangular: A^T x = b */
} sptrsv_op_t;

/* sptrsv_analyze for any of the four operators.  The paper treats the lower
 * triangle (Sec. II); the others are the same method on a mirrored system:
 * op(A) is brought on the device to the lower triangle L' that Sec. II's
 * forward substitution solves -- A^T by a CSR transpose (stable sort of the
 * entries by column), an upper triangle U by the exchange permutation P,
 * L' = P U P (so U x = b is L' (P x) = P b, the backward substitution).  The
 * analysis, the rewriting (Sec. III) and the solve then run on L', and the
 * solve structure is mirrored back once, so sptrsv_solve reads b and writes
 * x in A's row order with no extra copies.
 *   op       one of sptrsv_op_t (SPTRSV_ERR_INVALID_ARG otherwise).
 *   CSR      as for sptrsv_analyze; every row stores its diagonal, columns
 *            strictly ascending, A triangular in the sense op names.
 * Errors: SPTRSV_ERR_NOT_LOWER means an entry on the wrong side of the
 * diagonal for op (or a column outside [0, n)); the other validation codes
 * as for sptrsv_analyze.  Inspection calls (sptrsv_get_levels,
 * sptrsv_get_transformed) report rows and columns in A's numbering;
 * sptrsv_get_segments reports the levels of L'. */
SPTRSV_API sptrsv_status_t sptrsv_analyze_ex(int32_t n, int64_t nnz, const int32_t *d_row_ptr,
                                  const int32_t *d_col, const double *d_val, int32_t op,
                                  sptrsv_stream_t stream, sptrsv_plan_t *out);

/* Equation rewriting (Sec. III, Figs. 2-3): select rows (prm->select_mode),
 * compute on the device the fill of every candidate rewrite, the rewritten
 * coefficients and right-hand-side weights (FP64 always), assemble the
 * level-ordered solve structure and, for SPTRSV_SOLVE_AUTO, time candidate
 * launch configurations on it.  May be called again with other parameters;
 * SELECT_NONE restores the plain level sets. */
SPTRSV_API sptrsv_status_t sptrsv_transform(sptrsv_plan_t p, const sptrsv_transform_params_t *prm,
                                 sptrsv_stream_t stream);

/* x = op(A)^{-1} b (L^{-1} b for sptrsv_analyze's plans) for nrhs right-hand
 * sides (1..32 per launch; more are solved 32 columns at a time), row-major
 * [n][nrhs] device buffers.  x must not overlap b.  Asynchronous.  In F32_IR
 * precision the solve runs on FP32 copies of the values and refines with
 * FP64 residuals of the original matrix. */
SPTRSV_API sptrsv_status_t sptrsv_solve(sptrsv_plan_t p, const double *d_b, double *d_x,
                             int32_t nrhs, sptrsv_stream_t stream);

/* SPTRSV_SOLVE_AUTO keeps each tuned launch configuration in a process-wide
 * cache keyed by the device, the plan's shape (rows, entries, level sizes,
 * chosen segments, terms of the structure) and the requested constraints, so
 * a later transform of the same shape skips the timing.  This empties it. */
SPTRSV_API void sptrsv_autotune_cache_clear(void);

/* Synchronise `stream` and return the error latched by a kernel, if any. */
SPTRSV_API sptrsv_status_t sptrsv_check(sptrsv_plan_t p, sptrsv_stream_t stream);

SPTRSV_API sptrsv_status_t sptrsv_get_info(sptrsv_plan_t p, sptrsv_info_t *out);
SPTRSV_API void sptrsv_plan_destroy(sptrsv_plan_t p);

/* Analysis results (for inspection and tests), copied to device buffers:
 * level int32[n], level_ptr int32[nlev+1], perm int32[n] (rows ordered by
 * level, ascending row index inside a level; descending for an upper or
 * transposed-lower operator, whose mirrored triangle was analysed -- see
 * sptrsv_analyze_ex).  Any pointer may be NULL. */
SPTRSV_API sptrsv_status_t sptrsv_get_levels(sptrsv_plan_t p, int32_t *d_level,
                                  int32_t *d_level_ptr, int32_t *d_perm,
                                  sptrsv_stream_t stream);

/* The new levels chosen by the last transform as host arrays of
 * nlev_new entries: first original level t and number of absorbed levels d
 * (levels t..t+d form one new level). */
SPTRSV_API sptrsv_status_t sptrsv_get_segments(sptrsv_plan_t p, int32_t *h_first,
                                    int32_t *h_depth);

/* The transformed system in original row order (for inspection and tests).
 * Row i: x_i = (b_i - sum bw * b[bcol] - sum xval * x[xcol]) / diag_i.
 * Sizes: new_level int32[n], xptr/bptr int64[n+1], xcol/xval [nnz_x],
 * bcol/bw [nnz_b] (sptrsv_info_t).  Columns ascending inside a row. */
SPTRSV_API sptrsv_status_t sptrsv_get_transformed(sptrsv_plan_t p, int32_t *d_new_level,
                                       int64_t *d_xptr, int32_t *d_xcol,
                                       double *d_xval, int64_t *d_bptr,
                                       int32_t *d_bcol, double *d_bw,
                                       sptrsv_stream_t stream);

/* ---- Learned cost model ----------------------------------------------
 * The paper picks the rows to rewrite by hand (Sec. IV).  With a network
 * attached (sptrsv_set_costmodel, or the process-wide one of
 * sptrsv_costmodel_load), SPTRSV_SELECT_COSTMODEL predicts the log
 * solve time of every candidate rewrite from 17 features per candidate and
 * keeps the argmin; without one it falls back to heuristic H.  Candidates
 * (codes): d in {0,1,2,3,4,6,8} merges every d+1 levels (0 = plain level
 * sets); 100 + d in {108, 116} rewrites only the levels of fewer than 32
 * rows, up to d of them into the level before, within 4x the plain FLOPs
 * (heuristic H with those parameters).  sptrsv_info_t.chosen_depth is the
 * chosen code.  The network: F -> H -> H -> 1, ReLU, FP32, weights in one
 * flat array W1[F][H], b1[H], W2[H][H], b2[H], W3[H], b3 (row-major). */

/* Features of candidate codes (h_feat: [nd][17] floats, host; a code is
 * d in 0..16 or 100 + d with d in 0..16, SPTRSV_ERR_INVALID_ARG otherwise):
 *  0 log2 n, 1 log2 nnz, 2 dependencies per row, 3 log2 levels,
 *  4 log2 rows per level, 5-6 fraction of levels with < 32 / < 1024 rows,
 *  7 fraction of rows in levels of < 1024 rows, 8-11 fraction of rows with
 *  0 | 1-2 | 3-6 | >= 7 dependencies, 12 d, 13 log2 levels after merging,
 *  14 FLOPs after / FLOPs before, 15 fraction of rows rewritten, 16 1 for a
 *  thin-levels-only candidate, else 0.
 * Fill counts come from the device rewriting kernels; synchronises. */
SPTRSV_API sptrsv_status_t sptrsv_costmodel_features(sptrsv_plan_t p, const int32_t *h_depths,
                                                     int32_t nd, float *h_feat,
                                                     sptrsv_stream_t stream);
/* Attach (or detach with NULL) a network to a plan; not owned by the plan. */
SPTRSV_API sptrsv_status_t sptrsv_set_costmodel(sptrsv_plan_t p, sptrsv_mlp_t net);

SPTRSV_API int64_t sptrsv_mlp_num_params(int32_t n_in, int32_t hidden);
/* New network with the given initial weights (host array). */
SPTRSV_API sptrsv_status_t sptrsv_mlp_create(int32_t n_in, int32_t hidden,
                                             const float *h_params, sptrsv_mlp_t *out);
SPTRSV_API sptrsv_status_t sptrsv_mlp_get_params(sptrsv_mlp_t net, float *h_params);
/* Input normalisation used by SELECT_COSTMODEL: (f - mean) / std. */
SPTRSV_API sptrsv_status_t sptrsv_mlp_set_normalization(sptrsv_mlp_t net, const float *h_mean,
                                                        const float *h_std);
/* y[N] = network(X[N][F]) on device buffers (inputs already normalised). */
SPTRSV_API sptrsv_status_t sptrsv_mlp_forward(sptrsv_mlp_t net, const float *d_X, int32_t N,
                                              float *d_y, sptrsv_stream_t stream);
/* Gradients of mean((y - t)^2) w.r.t. all weights (flat, d_grads) and the
 * loss (d_loss); either output may be NULL. */
SPTRSV_API sptrsv_status_t sptrsv_mlp_grads(sptrsv_mlp_t net, const float *d_X,
                                            const float *d_target, int32_t N, float *d_grads,
                                            float *d_loss, sptrsv_stream_t stream);
/* One full-batch Adam step (beta1 0.9, beta2 0.999, eps 1e-8). */
SPTRSV_API sptrsv_status_t sptrsv_mlp_train_step(sptrsv_mlp_t net, const float *d_X,
                                                 const float *d_target, int32_t N, float lr,
                                                 float *d_loss, sptrsv_stream_t stream);
SPTRSV_API void sptrsv_mlp_destroy(sptrsv_mlp_t net);

/* Input normalisation computed by the library (training data stay on the
 * device; no host arithmetic): sptrsv_mlp_fit_normalization sets the
 * network's statistics to the column means and standard deviations of
 * d_X[N][F] (FP64 sums in a fixed order; a deviation below 1e-6 is taken as
 * 1) and synchronises `stream`; sptrsv_mlp_normalize writes
 * d_Xn = (d_X - mean) / std (d_Xn may equal d_X) and synchronises;
 * sptrsv_mlp_get_normalization copies the statistics out (mean 0, std 1
 * before any are set). */
SPTRSV_API sptrsv_status_t sptrsv_mlp_fit_normalization(sptrsv_mlp_t net, const float *d_X,
                                                        int32_t N, sptrsv_stream_t stream);
SPTRSV_API sptrsv_status_t sptrsv_mlp_normalize(sptrsv_mlp_t net, const float *d_X, int32_t N,
                                                float *d_Xn, sptrsv_stream_t stream);
SPTRSV_API sptrsv_status_t sptrsv_mlp_get_normalization(sptrsv_mlp_t net, float *h_mean,
                                                        float *h_std);

/* Network files.  Layout (little-endian): the 8 bytes "SPTRSVNN"; int32
 * version (1), F, H, has_normalisation; float32 weights (the flat layout
 * above, sptrsv_mlp_num_params(F, H) of them); float32 mean[F]; float32
 * std[F]; nothing after.  sptrsv_mlp_save writes a network (synchronises the
 * device copy of its weights); sptrsv_mlp_load creates a new network from a
 * file (SPTRSV_ERR_INVALID_ARG for a missing, short, long or foreign file).
 * Adam's moments are not saved: a loaded network trains from fresh moments. */
SPTRSV_API sptrsv_status_t sptrsv_mlp_save(sptrsv_mlp_t net, const char *path);
SPTRSV_API sptrsv_status_t sptrsv_mlp_load(const char *path, sptrsv_mlp_t *out);

/* The process-wide cost model: SPTRSV_SELECT_COSTMODEL uses a plan's own
 * network (sptrsv_set_costmodel) if attached, else this one, else heuristic
 * H.  sptrsv_costmodel_load reads a network file into it (owned by the
 * library, replacing and freeing an earlier loaded one); sptrsv_costmodel_save
 * writes it (SPTRSV_ERR_BAD_STATE when there is none);
 * sptrsv_costmodel_set_default makes a caller-owned network the default (NULL
 * clears it; destroying that network also clears it).  Not to be called
 * while a transform runs in another thread. */
SPTRSV_API sptrsv_status_t sptrsv_costmodel_load(const char *path);
SPTRSV_API sptrsv_status_t sptrsv_costmodel_save(const char *path);
SPTRSV_API sptrsv_status_t sptrsv_costmodel_set_default(sptrsv_mlp_t net);

/* The process-wide per-segment network of SPTRSV_SELECT_SEGMODEL (8 input
 * features, see sptrsv_segment_features), with the same ownership rules as
 * the cost model's; SPTRSV_ERR_INVALID_ARG for a network of another width. */
SPTRSV_API sptrsv_status_t sptrsv_segmodel_load(const char *path);
SPTRSV_API sptrsv_status_t sptrsv_segmodel_set_default(sptrsv_mlp_t net);

/* Features of every candidate segment of the analysed plan: for kept level
 * t (0 <= t < nlev) and depth d (0 <= d <= d_max <= 16), row t*(d_max+1)+d of
 * h_feat [nlev*(d_max+1)][8] holds log2(1 + rows), log2(1 + x and b terms),
 * log2(1 + most terms of a row), terms per row, d, fraction of rows
 * rewritten, log2 n and log2(nnz/n) of the segment merging levels t..t+d;
 * h_ok[t*(d_max+1)+d] = 1 where that segment exists within the fill cap
 * (max_row_fill of the last transform, 1024 before any).  Synchronises
 * `stream`. */
SPTRSV_API sptrsv_status_t sptrsv_segment_features(sptrsv_plan_t p, int32_t d_max,
                                                   float *h_feat, uint8_t *h_ok,
                                                   sptrsv_stream_t stream);

/* Time of each new level within a solve: `reps` solves of d_b into d_x
 * (one column), each stamping the completion of every chunk; h_us[g] = the
 * median over the solves of T(g) - T(g-1), T(g) the latest completion of a
 * chunk of new levels 0..g (T(-1) the solve's start), so that the times add
 * up to the solve.  Needs the staged synchronisation-free kernel (FP64, one
 * column, staging on, no single-CTA tail): SPTRSV_ERR_UNSUPPORTED otherwise.
 * Synchronises `stream`. */
SPTRSV_API sptrsv_status_t sptrsv_level_times(sptrsv_plan_t p, const double *d_b, double *d_x,
                                              int32_t reps, double *h_us,
                                              sptrsv_stream_t stream);

/* Batched solve (the paper treats one matrix; this serves many independent
 * systems of uneven size at once).  All plans must live on the current
 * device, be transformed with the same precision, and stay alive (and not be
 * transformed again) while the batch exists; at most as many plans as the
 * GPU holds co-resident CTAs (SPTRSV_ERR_UNSUPPORTED otherwise).  Refinement
 * tolerance, step limit (<= 16) and wait bound come from the first plan. */
SPTRSV_API sptrsv_status_t sptrsv_batch_create(const sptrsv_plan_t *plans, int32_t count,
                                               sptrsv_batch_t *out);

/* Solves every plan's system in ONE persistent launch: matrix i owns a group
 * of CTAs sized by its bytes, solves synchronisation-free inside the group
 * and separates the refinement phases (FP32 solve, FP64 residual, FP32
 * correction) with barriers on its own counter.  h_b / h_x are host arrays
 * of `count` device pointers to row-major [n_i, h_nrhs[i]] buffers
 * (1 <= h_nrhs[i] <= 32).  On a non-default stream the sequence is captured
 * in a CUDA graph on the first call and replayed afterwards (re-captured if
 * the scratch must grow); the first call, which may allocate, should come
 * before any stream capture of the caller's own.  Waits for the previous
 * batch_solve on this batch to finish before reusing its staging table. */
SPTRSV_API sptrsv_status_t sptrsv_batch_solve(sptrsv_batch_t batch, const double *const *h_b,
                                              double *const *h_x, const int32_t *h_nrhs,
                                              sptrsv_stream_t stream);

/* Synchronise `stream` and return an error a batch kernel latched. */
SPTRSV_API sptrsv_status_t sptrsv_batch_check(sptrsv_batch_t batch, sptrsv_stream_t stream);

/* After the last batch_solve completed: per matrix the refinement steps
 * applied, whether the tolerance was met, and the CTAs of its group; whether
 * the launch ran from a CUDA graph.  Any pointer may be NULL. */
SPTRSV_API sptrsv_status_t sptrsv_batch_get_info(sptrsv_batch_t batch, int32_t *h_iters,
                                                 int32_t *h_converged, int32_t *h_cta_count,
                                                 int32_t *h_graph);
/* Per matrix, the milliseconds its CTA group spent in the last batched solve
 * (first CTA in to last CTA out, %globaltimer); synchronises with that solve.
 * SPTRSV_ERR_BAD_STATE before any solve.  The groups are sized so that the
 * slowest matrix is as fast as it can be: the first solve with a set of
 * column counts runs once with groups predicted from each matrix's levels
 * and chunks per level, measures every group, and re-sizes the groups from
 * the measured times before the graph is captured (that first call solves
 * twice). */
SPTRSV_API sptrsv_status_t sptrsv_batch_get_times(sptrsv_batch_t b, float *h_ms);
SPTRSV_API void sptrsv_batch_destroy(sptrsv_batch_t batch);

/* Preconditioners of sptrsv_pcg_create, both built on A's lower triangle. */
typedef enum {
    SPTRSV_PRECOND_SGS = 0,  /* symmetric Gauss-Seidel: M = (D + L) D^{-1} (D + L)^T */
    SPTRSV_PRECOND_IC0 = 1   /* zero-fill incomplete Cholesky: M = C C^T */
} sptrsv_precond_t;

/* Preconditioned conjugate gradients -- a consumer of the triangular solve
 * (Sec. I names the iterative solvers that spend their time in SpTRSV as
 * the method's users).  For an SPD matrix A = L + D + L^T the preconditioner
 * is built on a lower triangle T with the pattern of D + L:
 *   SPTRSV_PRECOND_SGS  T = D + L,  M = T D^{-1} T^T;
 *   SPTRSV_PRECOND_IC0  T = C, the IC(0) factor (C C^T = A on the pattern of
 *                       D + L, row by row: C_ij = (A_ij - sum_k C_ik C_jk) /
 *                       C_jj over the k < j stored in both rows, C_ii =
 *                       sqrt(A_ii - sum_k C_ik^2)),  M = C C^T.
 * Each step applies M^{-1} as two triangular solves: T y = r, then
 * T^T z = D y (SGS) or T^T z = y (IC(0)).
 *
 * sptrsv_pcg_create: A is the FULL symmetric matrix in device CSR
 * (row_ptr[n+1], col[nnz], val[nnz], int32 / FP64, columns ascending per
 * row, diagonal stored, n >= 1, nnz >= 1); the library copies it, so the
 * caller's arrays may be freed afterwards.  The call extracts D + L on the
 * device, for IC(0) factors it (one launch per level of D + L's dependency
 * DAG), and builds two plans of T, one analysed as SPTRSV_OP_LOWER and one as
 * SPTRSV_OP_LOWER_TRANS, transformed with prm_lower and prm_upper (NULL:
 * sptrsv_default_params).  The PCG object owns both plans; synchronises
 * `stream`.  The library does not check that A is symmetric or positive
 * definite; the iteration has no meaning otherwise.
 * Errors: SPTRSV_ERR_INVALID_ARG (null pointer, sizes, unknown precond),
 * SPTRSV_ERR_UNSORTED (row_ptr not monotone inside [0, nnz]),
 * SPTRSV_ERR_NOT_LOWER (a column outside [0, n)), the analysis codes of
 * D + L (unsorted columns, missing or zero diagonal), SPTRSV_ERR_ZERO_DIAG
 * also for an IC(0) pivot <= 0 (the incomplete factorisation breaks down),
 * the transforms' codes, SPTRSV_ERR_OOM, SPTRSV_ERR_CUDA.
 *
 * sptrsv_pcg_get_plans: the two plans (borrowed: valid until
 * sptrsv_pcg_destroy) for sptrsv_get_info, profiling or a new transform.
 *
 * sptrsv_pcg_get_factor: *h_nnz = entries of T; if d_val is not NULL, copies
 * T's values (device, FP64, h_nnz) in the order of A's lower-triangle
 * entries (row by row, columns ascending) on `stream`, asynchronously.
 *
 * sptrsv_pcg_solve: x (device, FP64, n) holds the initial guess on entry and
 * the iterate on return; b (device, FP64, n) is not modified.  Steps until
 * |r|_2 <= rtol |b|_2 for the recursively updated residual r, or max_iter
 * steps; *h_iters gets the steps taken and *h_relres |r|_2 / |b|_2 at the
 * end (either pointer may be NULL).  b = 0 gives x = 0 and no step.  Reads
 * the residual norm to the host once per step, so the call synchronises
 * `stream` every step and returns after the solve is complete.  Dot products
 * reduce in a fixed order; a synchronisation-free triangular solve adds a
 * row's terms partly in the order they become ready, so two runs can differ
 * in the last bits (and, near the tolerance, by one step).  A latched
 * error of either plan's solves (e.g. SPTRSV_ERR_TIMEOUT) is returned at the
 * end; calls on one PCG object must not overlap.  Errors:
 * SPTRSV_ERR_INVALID_ARG (null object, b or x, max_iter < 0, rtol < 0 or
 * NaN, a b whose norm is not finite), SPTRSV_ERR_BREAKDOWN (the starting
 * residual b - A x0 is not finite, e.g. a NaN in x0; or a step met (p, A p)
 * <= 0 or not finite, e.g. an indefinite A, or a residual that is not
 * finite; x is then left in an unspecified state and *h_iters / *h_relres
 * describe the step that failed), SPTRSV_ERR_CUDA, and the solves'. */
SPTRSV_API sptrsv_status_t sptrsv_pcg_create(int32_t n, int64_t nnz, const int32_t *d_row_ptr,
                                             const int32_t *d_col, const double *d_val,
                                             int32_t precond,
                                             const sptrsv_transform_params_t *prm_lower,
                                             const sptrsv_transform_params_t *prm_upper,
                                             sptrsv_stream_t stream, sptrsv_pcg_t *out);
SPTRSV_API sptrsv_status_t sptrsv_pcg_get_plans(sptrsv_pcg_t pcg, sptrsv_plan_t *lower,
                                                sptrsv_plan_t *upper);
SPTRSV_API sptrsv_status_t sptrsv_pcg_get_factor(sptrsv_pcg_t pcg, int64_t *h_nnz,
                                                 double *d_val, sptrsv_stream_t stream);
SPTRSV_API sptrsv_status_t sptrsv_pcg_solve(sptrsv_pcg_t pcg, const double *d_b, double *d_x,
                                            double rtol, int32_t max_iter, int32_t *h_iters,
                                            double *h_relres, sptrsv_stream_t stream);
SPTRSV_API void sptrsv_pcg_destroy(sptrsv_pcg_t pcg);

/* The FP32 + FP64-refinement solve without any device allocation.  The
 * paper has no counterpart: this exists for callers that cannot call
 * cudaMalloc when they solve -- code recording a CUDA graph, applications
 * whose device memory comes from their own pool or is fixed at start-up,
 * loops that must not synchronise the device.  sptrsv_solve in SPTRSV_F32_IR
 * precision allocates its two scratch arrays (FP32 correction, FP64
 * residual) on first use of a size; this call takes them instead from one
 * file-scope __device__ array of 12 MiB that every GPU loading the library
 * holds until the process exits.
 *  - The plan must have been transformed with precision SPTRSV_F32_IR
 *    (SPTRSV_ERR_BAD_STATE otherwise); b and x as for sptrsv_solve.
 *  - n * nrhs must not exceed 1,048,576 (SPTRSV_ERR_UNSUPPORTED otherwise).
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) once; make that first call before any stream
 *    capture.
 *  - All calls, on every plan and stream, share the one array: calls that
 *    overlap on the GPU race and give wrong results.  Nothing in it needs to
 *    start at zero; it keeps whatever the last call left.
 *  - Asynchronous like sptrsv_solve; errors found by kernels are latched in
 *    the plan and returned by sptrsv_check. */
SPTRSV_API sptrsv_status_t sptrsv_solve_ir_noalloc(sptrsv_plan_t p, const double *d_b,
                                                   double *d_x, int32_t nrhs,
                                                   sptrsv_stream_t stream);

/* Profiling (not part of the paper's method): while enabled, sptrsv_solve
 * records CUDA events on its stream around its solve kernel launch(es)
 * (FP64 only).
 * sptrsv_last_kernel_ms waits for the last solve's end event and returns the
 * elapsed milliseconds; SPTRSV_ERR_BAD_STATE if no profiled solve ran. */
SPTRSV_API sptrsv_status_t sptrsv_set_profiling(sptrsv_plan_t p, int32_t on);
SPTRSV_API sptrsv_status_t sptrsv_last_kernel_ms(sptrsv_plan_t p, float *ms);

/* Test hook for failure detection (not part of the paper's method): makes
 * row `row` of the current solve structure read its own unknown, a wait no
 * write can ever satisfy.  A later synchronisation-free solve must then give
 * up after wait_timeout_ms and sptrsv_check must return SPTRSV_ERR_TIMEOUT;
 * the plan is unusable afterwards.  The row must have at least one
 * off-diagonal term (SPTRSV_ERR_UNSUPPORTED otherwise).  The single-CTA tail
 * (tail_rows) is dropped and stays off for the plan's life (the tail kernel
 * does not wait), so every level runs in the main kernel.  A later
 * sptrsv_transform rebuilds the structure from the matrix, which removes
 * the injected dependency. */
SPTRSV_API sptrsv_status_t sptrsv_debug_inject_wait(sptrsv_plan_t p, int32_t row);

/* Per-level features of the analysis (the matrix-analysis module, Sec. IV),
 * h_feat [nlev][11 + lifts] floats (host), for level l:
 *   0 rows, 1 off-diagonal entries of its rows,
 *   2..9 rows by off-diagonal count c in log2 bins: bin 0 c = 0, bin b
 *        (1..6) 2^(b-1) <= c < 2^b, bin 7 c >= 64,
 *   10 ancestor span: max over its rows of l - (lowest level it depends on),
 *   10 + r (r = 1..lifts) FLOPs added when every row of l is rewritten to
 *        target level l - r (2 per added x or b term), -1 when a row would
 *        exceed max_row_fill, 0 when l < r.
 * Counted on the device (the fill columns by the rewriting kernels);
 * synchronises `stream`.  lifts in 0..16. */
SPTRSV_API sptrsv_status_t sptrsv_level_features(sptrsv_plan_t p, int32_t lifts,
                                                 float *h_feat, sptrsv_stream_t stream);

/* Weighted critical path of the plan's current FP64 solve structure (the
 * system the solve kernels run, rewritten rows included): CP = max over rows
 * of f(i) = hop_weight + terms(i) + max f(j) over the unknowns j its x terms
 * read, terms(i) = its x terms plus b terms (hop_weight <= 0: 16).  Computed
 * on the device one new level per launch; synchronises `stream`.
 * SPTRSV_ERR_BAD_STATE before the structure exists. */
SPTRSV_API sptrsv_status_t sptrsv_critical_path(sptrsv_plan_t p, int32_t hop_weight,
                                                int64_t *h_cp, sptrsv_stream_t stream);

/* Source of the kernel generated for tail segment `seg` (0-based, solve
 * order) of the plan's current configuration (codegen_rows, Sec. IV's
 * specialised code): the CUDA C++ text the runtime compiler was given, so
 * that a caller can see the matrix's row ids, unknown slots and
 * coefficients written into it.  Writes at most `cap` bytes including the
 * terminating zero into `buf` (host, may be null when cap is 0) and the full
 * length without the zero into *len.  SPTRSV_ERR_BAD_STATE when the segment
 * has no generated kernel, SPTRSV_ERR_INVALID_ARG for a bad segment index or
 * a null `len`. */
SPTRSV_API sptrsv_status_t sptrsv_codegen_source(sptrsv_plan_t p, int32_t seg, char *buf,
                                                 size_t cap, size_t *len);

/* The same generator on a segment's records given on the host (no plan, no
 * GPU): nrows rows in solve order grouped into nlev levels, K term slots per
 * row; h_row[p] the row index x is written to; h_nn[p] the term count (bits
 * 0-7), the mask of terms read from x (bits 8-23; a segment with any is not
 * generated) and 1 << 30 for a row whose coefficients are not divided by
 * its diagonal; h_term[4 (k nrows + p) + 0..3] = (slot q < p of an earlier
 * row of the segment, 0, low and high 32 bits of the coefficient);
 * h_diag[2p] = L_ii (used by undivided rows).  Output as for
 * sptrsv_codegen_source; SPTRSV_ERR_BAD_STATE when the segment would get no
 * kernel (not thin: 16 or more terms per level on average),
 * SPTRSV_ERR_INVALID_ARG for a slot that is not an earlier row. */
SPTRSV_API sptrsv_status_t sptrsv_codegen_source_from_records(
    int32_t nrows, int32_t K, int32_t nlev, const int32_t *h_row, const int32_t *h_nn,
    const int32_t *h_term, const double *h_diag, char *buf, size_t cap, size_t *len);

#ifdef __cplusplus
}
#endif
#endif /* SPTRSV_H */
