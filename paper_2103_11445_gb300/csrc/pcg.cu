// Preconditioned conjugate gradients for an SPD matrix A = L + D + L^T with
// one of two preconditioners built on A's lower triangle:
//   symmetric Gauss-Seidel  M = (D + L) D^{-1} (D + L)^T,
//   IC(0)                   M = C C^T, C the zero-fill incomplete Cholesky
//                           factor (the pattern of D + L, C C^T = A there).
// The triangular solve is the kernel of such preconditioners (Sec. I names
// iterative solvers as SpTRSV's consumers): every step applies M^{-1} as two
// of this library's solves -- T y = r on a plan of the triangle T (D + L or
// C), T^T z = D y (SGS) or T^T z = y (IC(0)) on a plan of the same triangle as
// SPTRSV_OP_LOWER_TRANS -- each analysed, rewritten (Sec. III) and tuned once,
// when the PCG object is created.  The IC(0) factor itself is computed level
// by level over the same dependency DAG the solve uses (row i needs the rows
// of its pattern, Sec. II's DAG_L), one launch per level.
//
// The vector work (A p, dot products, updates) runs in the kernels below;
// scalars (alpha, beta, the residual norm) stay on the device, and the host
// reads one number per step to test convergence.  Dot products reduce in a
// fixed order (per-block partial sums, then one block).
#include <cmath>
#include <vector>

#include "kernels.cuh"
#include "plan.cuh"

namespace sptrsv {

// the loop's scalars, kept on the device; rr and bb adjacent (read together)
struct PcgScalars {
    double rz;      // (r, z)
    double rz_new;
    double pq;      // (p, A p)
    double rr;      // (r, r)
    double bb;      // (b, b)
};

namespace {

constexpr int kDotBlocks = 1024;
constexpr int kDotThreads = 256;
constexpr int kSpmvLanes = 4;   // lanes per row of the matrix-vector product

// y = A x, or y = b - A x when b is given; kSpmvLanes lanes per row summing
// their entries in storage order, then a fixed shuffle tree.
__global__ void spmv_kernel(int32_t n, const int32_t *__restrict__ rp,
                            const int32_t *__restrict__ col, const double *__restrict__ val,
                            const double *__restrict__ x, const double *__restrict__ b,
                            double *__restrict__ y) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = t / kSpmvLanes;
    const int s = (int)(t % kSpmvLanes);
    double acc = 0.0;
    if (row < n) {
        const int32_t a = rp[row], e = rp[row + 1];
        for (int32_t k = a + s; k < e; k += kSpmvLanes) acc = fma(val[k], x[col[k]], acc);
    }
#pragma unroll
    for (int o = kSpmvLanes / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL_MASK, acc, o);
    if (row < n && s == 0) y[row] = b ? b[row] - acc : acc;
}

// Per-block partial sums of u . v over a fixed partition of [0, n).
__global__ void dot_partial_kernel(int32_t n, const double *__restrict__ u,
                                   const double *__restrict__ v, double *__restrict__ part) {
    __shared__ double sh[kDotThreads];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        s = fma(u[i], v[i], s);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = kDotThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// The partials summed in a fixed order into *out.
__global__ void dot_final_kernel(const double *__restrict__ part, double *out) {
    __shared__ double sh[kDotThreads];
    double s = 0.0;
    for (int i = threadIdx.x; i < kDotBlocks; i += kDotThreads) s += part[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = kDotThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// x += alpha p, r -= alpha q, alpha = rz / pq
__global__ void update_xr_kernel(int32_t n, const PcgScalars *sc, const double *__restrict__ p,
                                 const double *__restrict__ q, double *__restrict__ x,
                                 double *__restrict__ r) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double alpha = sc->rz / sc->pq;
    x[i] = fma(alpha, p[i], x[i]);
    r[i] = fma(-alpha, q[i], r[i]);
}

// p = z + beta p, beta = rz_new / rz (first step: p = z)
__global__ void update_p_kernel(int32_t n, const PcgScalars *sc, const double *__restrict__ z,
                                double *__restrict__ p, int first) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    p[i] = first ? z[i] : fma(sc->rz_new / sc->rz, p[i], z[i]);
}

__global__ void roll_rz_kernel(PcgScalars *sc) { sc->rz = sc->rz_new; }

// w = D y with D the diagonal of A
__global__ void scale_kernel(int32_t n, const double *__restrict__ d, const double *__restrict__ y,
                             double *__restrict__ w) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w[i] = d[i] * y[i];
}

// entries of row i with column <= i (A's lower triangle D + L)
__global__ void tril_count_kernel(int32_t n, const int32_t *__restrict__ rp,
                                  const int32_t *__restrict__ col, int32_t *__restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t c = 0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) c += col[k] <= i;
    cnt[i] = c;
}

__global__ void tril_gather_kernel(int32_t n, const int32_t *__restrict__ rp,
                                   const int32_t *__restrict__ col, const double *__restrict__ val,
                                   const int32_t *__restrict__ lrp, int32_t *__restrict__ lcol,
                                   double *__restrict__ lval) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t o = lrp[i];
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
        if (col[k] <= i) {
            lcol[o] = col[k];
            lval[o++] = val[k];
        }
}

// IC(0), rows of one level (their dependencies all lie in earlier levels):
// row i, columns j < i ascending, C_ij = (A_ij - sum_k C_ik C_jk) / C_jj over
// the k < j stored in both rows (a merge of two sorted column lists), then
// C_ii = sqrt(A_ii - sum_k C_ik^2).  c holds A's values on entry and C's on
// return.  A pivot <= 0 records the row in *err (atomicMin) and stores 1 so
// that later rows stay finite.
__global__ void ic0_level_kernel(const int32_t *__restrict__ rows, int32_t count,
                                 const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                 double *__restrict__ c, int32_t *err) {
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int32_t i = rows[t];
    const int32_t a = rp[i], e = rp[i + 1] - 1;   // e: the diagonal, last in the row
    double sq = 0.0;
    for (int32_t p = a; p < e; ++p) {
        const int32_t j = col[p];
        const int32_t jb = rp[j], je = rp[j + 1] - 1;
        double s = c[p];
        int32_t q = a, r = jb;
        while (q < p && r < je) {
            const int32_t cq = col[q], cr = col[r];
            if (cq == cr) {
                s = fma(-c[q], c[r], s);
                ++q;
                ++r;
            } else if (cq < cr) {
                ++q;
            } else {
                ++r;
            }
        }
        const double v = s / c[je];
        c[p] = v;
        sq = fma(v, v, sq);
    }
    const double d = c[e] - sq;
    if (d > 0.0) {
        c[e] = sqrt(d);
    } else {
        atomicMin(err, i);
        c[e] = 1.0;
    }
}

// the diagonal of A (0 where a row stores none)
__global__ void diag_kernel(int32_t n, const int32_t *__restrict__ rp,
                            const int32_t *__restrict__ col, const double *__restrict__ val,
                            double *__restrict__ d) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
        if (col[k] == i) v = val[k];
    d[i] = v;
}

unsigned blocks(int64_t count, int threads) { return (unsigned)((count + threads - 1) / threads); }

}  // namespace
}  // namespace sptrsv

using namespace sptrsv;

struct sptrsv_pcg_s {
    int32_t n = 0;
    int64_t nnz = 0;
    int32_t precond = SPTRSV_PRECOND_SGS;
    int32_t nnz_tri = 0;                             // entries of the triangle T
    sptrsv_plan_t lower = nullptr, upper = nullptr;   // owned
    DevArr<int32_t> rp, col;
    DevArr<double> val, tri_val, diag, r, z, p, q, y, part;
    DevArr<PcgScalars> sc;
    ~sptrsv_pcg_s() {
        sptrsv_plan_destroy(lower);
        sptrsv_plan_destroy(upper);
    }
};

namespace {

#define PCK(x)                                                                 \
    do {                                                                       \
        cudaError_t _e = (x);                                                  \
        if (_e != cudaSuccess) {                                               \
            (void)cudaGetLastError();                                          \
            return _e == cudaErrorMemoryAllocation ? SPTRSV_ERR_OOM : SPTRSV_ERR_CUDA; \
        }                                                                      \
    } while (0)

sptrsv_status_t dot(sptrsv_pcg_t g, const double *u, const double *v, double *out,
                    cudaStream_t s) {
    dot_partial_kernel<<<kDotBlocks, kDotThreads, 0, s>>>(g->n, u, v, g->part.p);
    dot_final_kernel<<<1, kDotThreads, 0, s>>>(g->part.p, out);
    PCK(cudaGetLastError());
    return SPTRSV_OK;
}

// z = M^{-1} r: T y = r, then T^T z = D y (SGS) or T^T z = y (IC(0))
sptrsv_status_t precond_apply(sptrsv_pcg_t g, const double *r, double *z, cudaStream_t s) {
    sptrsv_status_t st = sptrsv_solve(g->lower, r, g->y.p, 1, s);
    if (st != SPTRSV_OK) return st;
    if (g->precond == SPTRSV_PRECOND_IC0) return sptrsv_solve(g->upper, g->y.p, z, 1, s);
    scale_kernel<<<blocks(g->n, 256), 256, 0, s>>>(g->n, g->diag.p, g->y.p, g->q.p);
    PCK(cudaGetLastError());
    return sptrsv_solve(g->upper, g->q.p, z, 1, s);
}

// C = IC(0) of the SPD matrix whose lower triangle is (lrp, lcol, c): levels
// from an analysis of the triangle, then one launch per level.
sptrsv_status_t ic0_factor(int32_t n, int32_t nnz_l, const int32_t *lrp, const int32_t *lcol,
                           double *c, sptrsv_stream_t stream) {
    cudaStream_t s = (cudaStream_t)stream;
    sptrsv_plan_t tmp = nullptr;
    sptrsv_status_t st = sptrsv_analyze(n, nnz_l, lrp, lcol, c, stream, &tmp);
    if (st != SPTRSV_OK) return st;
    struct Guard {
        sptrsv_plan_t p;
        ~Guard() { sptrsv_plan_destroy(p); }
    } guard{tmp};
    sptrsv_info_t info;
    if ((st = sptrsv_get_info(tmp, &info)) != SPTRSV_OK) return st;
    DevArr<int32_t> perm, lptr, err;
    PCK(perm.alloc(n));
    PCK(lptr.alloc((size_t)info.nlev + 1));
    PCK(err.alloc(1));
    if ((st = sptrsv_get_levels(tmp, nullptr, lptr.p, perm.p, stream)) != SPTRSV_OK) return st;
    std::vector<int32_t> h((size_t)info.nlev + 1);
    PCK(cudaMemcpyAsync(h.data(), lptr.p, h.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PCK(cudaMemsetAsync(err.p, 0x7f, sizeof(int32_t), s));
    PCK(cudaStreamSynchronize(s));
    for (int32_t l = 0; l < info.nlev; ++l) {
        const int32_t cnt = h[l + 1] - h[l];
        ic0_level_kernel<<<blocks(cnt, 128), 128, 0, s>>>(perm.p + h[l], cnt, lrp, lcol, c,
                                                          err.p);
    }
    PCK(cudaGetLastError());
    int32_t bad = 0;
    PCK(cudaMemcpyAsync(&bad, err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PCK(cudaStreamSynchronize(s));
    return bad == 0x7f7f7f7f ? SPTRSV_OK : SPTRSV_ERR_ZERO_DIAG;
}

}  // namespace

extern "C" {

sptrsv_status_t sptrsv_pcg_create(int32_t n, int64_t nnz, const int32_t *d_row_ptr,
                                  const int32_t *d_col, const double *d_val, int32_t precond,
                                  const sptrsv_transform_params_t *prm_lower,
                                  const sptrsv_transform_params_t *prm_upper,
                                  sptrsv_stream_t stream, sptrsv_pcg_t *out) {
    if (!out) return SPTRSV_ERR_INVALID_ARG;
    *out = nullptr;
    if (n <= 0 || nnz <= 0 || nnz > INT32_MAX || !d_row_ptr || !d_col || !d_val)
        return SPTRSV_ERR_INVALID_ARG;
    if (precond != SPTRSV_PRECOND_SGS && precond != SPTRSV_PRECOND_IC0)
        return SPTRSV_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    sptrsv_pcg_s *g = new sptrsv_pcg_s();
    sptrsv_status_t st = SPTRSV_OK;
    auto fail = [&](sptrsv_status_t e) {
        delete g;
        return e;
    };
#define PCKC(x)                                                                \
    do {                                                                       \
        cudaError_t _e = (x);                                                  \
        if (_e != cudaSuccess) {                                               \
            (void)cudaGetLastError();                                          \
            return fail(_e == cudaErrorMemoryAllocation ? SPTRSV_ERR_OOM : SPTRSV_ERR_CUDA); \
        }                                                                      \
    } while (0)
    g->n = n;
    g->nnz = nnz;
    g->precond = precond;
    PCKC(g->rp.alloc((size_t)n + 1));
    PCKC(g->col.alloc(nnz));
    PCKC(g->val.alloc(nnz));
    for (DevArr<double> *v : {&g->diag, &g->r, &g->z, &g->p, &g->q, &g->y}) PCKC(v->alloc(n));
    PCKC(g->part.alloc(kDotBlocks));
    PCKC(g->sc.alloc(1));
    PCKC(cudaMemcpyAsync(g->rp.p, d_row_ptr, ((size_t)n + 1) * sizeof(int32_t),
                         cudaMemcpyDeviceToDevice, s));
    PCKC(cudaMemcpyAsync(g->col.p, d_col, nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    PCKC(cudaMemcpyAsync(g->val.p, d_val, nnz * sizeof(double), cudaMemcpyDeviceToDevice, s));
    {   // A's structure: row_ptr monotone in [0, nnz], columns in [0, n)
        DevArr<unsigned long long> err;
        PCKC(err.alloc(1));
        PCKC(cudaMemsetAsync(err.p, 0xff, sizeof(unsigned long long), s));
        PCKC(launch_csr_check(n, nnz, g->rp.p, g->col.p, err.p, s));
        unsigned long long h = 0;
        PCKC(cudaMemcpyAsync(&h, err.p, sizeof(h), cudaMemcpyDeviceToHost, s));
        PCKC(cudaStreamSynchronize(s));
        if (h != ~0ull) return fail((sptrsv_status_t)(h & 0xff));
    }
    diag_kernel<<<blocks(n, 256), 256, 0, s>>>(n, g->rp.p, g->col.p, g->val.p, g->diag.p);
    PCKC(cudaGetLastError());
    {   // the triangle T (D + L, or its IC(0) factor), analysed as the forward
        // and as the transposed operator
        DevArr<int32_t> cnt, lrp, lcol;
        DevArr<int64_t> tmp;
        PCKC(cnt.alloc(n));
        PCKC(lrp.alloc((size_t)n + 1));
        PCKC(tmp.alloc(scan_tmp_elems(n)));
        tril_count_kernel<<<blocks(n, 256), 256, 0, s>>>(n, g->rp.p, g->col.p, cnt.p);
        PCKC(cudaGetLastError());
        PCKC(exclusive_scan_i32_i32(cnt.p, lrp.p, n, tmp.p, s));
        int32_t nnz_l = 0;
        PCKC(cudaMemcpyAsync(&nnz_l, lrp.p + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PCKC(cudaStreamSynchronize(s));
        if (nnz_l <= 0) return fail(SPTRSV_ERR_MISSING_DIAG);
        g->nnz_tri = nnz_l;
        PCKC(lcol.alloc(nnz_l));
        PCKC(g->tri_val.alloc(nnz_l));
        double *tv = g->tri_val.p;
        tril_gather_kernel<<<blocks(n, 256), 256, 0, s>>>(n, g->rp.p, g->col.p, g->val.p, lrp.p,
                                                          lcol.p, tv);
        PCKC(cudaGetLastError());
        if (precond == SPTRSV_PRECOND_IC0 &&
            (st = ic0_factor(n, nnz_l, lrp.p, lcol.p, tv, stream)) != SPTRSV_OK)
            return fail(st);
        if ((st = sptrsv_analyze_ex(n, nnz_l, lrp.p, lcol.p, tv, SPTRSV_OP_LOWER, stream,
                                    &g->lower)) != SPTRSV_OK ||
            (st = sptrsv_analyze_ex(n, nnz_l, lrp.p, lcol.p, tv, SPTRSV_OP_LOWER_TRANS,
                                    stream, &g->upper)) != SPTRSV_OK)
            return fail(st);
        PCKC(cudaStreamSynchronize(s));
    }
    sptrsv_transform_params_t dflt;
    sptrsv_default_params(&dflt);
    if ((st = sptrsv_transform(g->lower, prm_lower ? prm_lower : &dflt, stream)) != SPTRSV_OK ||
        (st = sptrsv_transform(g->upper, prm_upper ? prm_upper : &dflt, stream)) != SPTRSV_OK)
        return fail(st);
#undef PCKC
    *out = g;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_pcg_get_plans(sptrsv_pcg_t g, sptrsv_plan_t *lower, sptrsv_plan_t *upper) {
    if (!g) return SPTRSV_ERR_INVALID_ARG;
    if (lower) *lower = g->lower;
    if (upper) *upper = g->upper;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_pcg_get_factor(sptrsv_pcg_t g, int64_t *h_nnz, double *d_val,
                                      sptrsv_stream_t stream) {
    if (!g) return SPTRSV_ERR_INVALID_ARG;
    if (h_nnz) *h_nnz = g->nnz_tri;
    if (d_val) {
        cudaStream_t s = (cudaStream_t)stream;
        PCK(cudaMemcpyAsync(d_val, g->tri_val.p, (size_t)g->nnz_tri * sizeof(double),
                            cudaMemcpyDeviceToDevice, s));
    }
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_pcg_solve(sptrsv_pcg_t g, const double *d_b, double *d_x, double rtol,
                                 int32_t max_iter, int32_t *h_iters, double *h_relres,
                                 sptrsv_stream_t stream) {
    if (!g || max_iter < 0 || !(rtol >= 0.0)) return SPTRSV_ERR_INVALID_ARG;
    if (h_iters) *h_iters = 0;
    if (h_relres) *h_relres = 0.0;
    const int32_t n = g->n;
    if (n == 0) return SPTRSV_OK;
    if (!d_b || !d_x) return SPTRSV_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    PcgScalars *sc = g->sc.p;
    const unsigned vb = blocks(n, 256);
    const unsigned sb = blocks((int64_t)n * kSpmvLanes, 256);
    sptrsv_status_t st;
    // r = b - A x, z = M^{-1} r, p = z, rz = (r, z), bb = (b, b)
    spmv_kernel<<<sb, 256, 0, s>>>(n, g->rp.p, g->col.p, g->val.p, d_x, d_b, g->r.p);
    PCK(cudaGetLastError());
    if ((st = dot(g, d_b, d_b, &sc->bb, s)) != SPTRSV_OK) return st;
    if ((st = dot(g, g->r.p, g->r.p, &sc->rr, s)) != SPTRSV_OK) return st;
    double host[2];
    PCK(cudaMemcpyAsync(host, &sc->rr, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    PCK(cudaStreamSynchronize(s));
    const double bnorm = std::sqrt(host[1]);
    if (!std::isfinite(bnorm)) return SPTRSV_ERR_INVALID_ARG;   // b holds a NaN or an infinity
    if (bnorm == 0.0) {   // b = 0: the solution is x = 0
        PCK(cudaMemsetAsync(d_x, 0, (size_t)n * sizeof(double), s));
        PCK(cudaStreamSynchronize(s));
        return SPTRSV_OK;
    }
    double rel = std::sqrt(host[0]) / bnorm;
    int32_t it = 0;
    // a NaN or an infinity in x0 (or in A): both rel > rtol and rel <= rtol
    // would be false, and the loop would end at once with a garbage x
    if (!std::isfinite(rel)) {
        if (h_relres) *h_relres = rel;
        return SPTRSV_ERR_BREAKDOWN;
    }
    if (rel > rtol) {
        if ((st = precond_apply(g, g->r.p, g->z.p, s)) != SPTRSV_OK) return st;
        update_p_kernel<<<vb, 256, 0, s>>>(n, sc, g->z.p, g->p.p, 1);
        PCK(cudaGetLastError());
        if ((st = dot(g, g->r.p, g->z.p, &sc->rz, s)) != SPTRSV_OK) return st;
    }
    while (it < max_iter && rel > rtol) {
        spmv_kernel<<<sb, 256, 0, s>>>(n, g->rp.p, g->col.p, g->val.p, g->p.p, nullptr, g->q.p);
        PCK(cudaGetLastError());
        if ((st = dot(g, g->p.p, g->q.p, &sc->pq, s)) != SPTRSV_OK) return st;
        update_xr_kernel<<<vb, 256, 0, s>>>(n, sc, g->p.p, g->q.p, d_x, g->r.p);
        PCK(cudaGetLastError());
        ++it;
        if ((st = dot(g, g->r.p, g->r.p, &sc->rr, s)) != SPTRSV_OK) return st;
        double pq_rr[2] = {0, 0};   // (p, A p) and (r, r) are adjacent
        PCK(cudaMemcpyAsync(pq_rr, &sc->pq, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        PCK(cudaStreamSynchronize(s));
        rel = std::sqrt(pq_rr[1]) / bnorm;
        // breakdown: an indefinite A (or preconditioner) gives (p, A p) <= 0,
        // and any non-finite value would otherwise end the loop as if converged
        if (!(pq_rr[0] > 0.0) || !std::isfinite(pq_rr[0]) || !std::isfinite(rel)) {
            if (h_iters) *h_iters = it;
            if (h_relres) *h_relres = rel;
            return SPTRSV_ERR_BREAKDOWN;
        }
        if (rel <= rtol || it >= max_iter) break;
        if ((st = precond_apply(g, g->r.p, g->z.p, s)) != SPTRSV_OK) return st;
        if ((st = dot(g, g->r.p, g->z.p, &sc->rz_new, s)) != SPTRSV_OK) return st;
        update_p_kernel<<<vb, 256, 0, s>>>(n, sc, g->z.p, g->p.p, 0);
        roll_rz_kernel<<<1, 1, 0, s>>>(sc);
        PCK(cudaGetLastError());
    }
    if ((st = sptrsv_check(g->lower, s)) != SPTRSV_OK) return st;
    if ((st = sptrsv_check(g->upper, s)) != SPTRSV_OK) return st;
    if (h_iters) *h_iters = it;
    if (h_relres) *h_relres = rel;
    return SPTRSV_OK;
}

void sptrsv_pcg_destroy(sptrsv_pcg_t g) { delete g; }

}  // extern "C"
