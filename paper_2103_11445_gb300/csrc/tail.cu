// Single-CTA tail of the solve: a GPU form of two things Sec. IV leaves
// open -- packing short levels together, and taking indirect indexing off
// the path of thin levels (the paper's code generator bakes indices in as
// constants; here each thread's records are loaded ahead of need instead).
#include "tail.cuh"

#include "plan.cuh"

namespace sptrsv {
namespace {

// Division by the diagonal, the same steps as the solve kernels take: with
// y = RN(1/d) precomputed (0 when d lies outside the safe range), q = RN(s y)
// is within an ulp of s/d, the remainder r = s - d q is exact (one FMA), and
// RN(q + r y) is the correctly rounded quotient (Markstein, IBM J. Res. Dev.
// 1990) while |s| lies in [2^-900, 2^900) and |q| in [2^-1000, 2^1000) (bit
// patterns compared as integers); anything else takes an IEEE division.
__device__ __forceinline__ double div_diag(double s, double d, double y) {
    constexpr unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull;
    constexpr unsigned long long kSlo = 0x07B0000000000000ull, kShi = 0x7830000000000000ull;
    constexpr unsigned long long kQlo = 0x0170000000000000ull, kQhi = 0x7E70000000000000ull;
    const unsigned long long as = (unsigned long long)__double_as_longlong(s) & kAbs;
    if (__double_as_longlong(y) != 0 && as - kSlo < kShi - kSlo) {
        const double q = s * y;
        const double r = fma(-q, d, s);
        const double q2 = fma(r, y, q);
        const unsigned long long a = (unsigned long long)__double_as_longlong(q2) & kAbs;
        if (a - kQlo < kQhi - kQlo) return q2;
    }
    return s / d;
}

// Runs of levels at the end of the order that are at most one CTA wide are
// solved by one CTA each (a segment): level l's rows go to threads 0..w-1
// with __syncthreads between levels, so a dependency hop stays inside one SM
// (a shared-memory store and a barrier instead of a store's flight to L2 and
// a remote poll).  Before each segment, tail_const_kernel folds every term
// that reads no unknown of the segment (b terms of rewritten rows, unknowns
// solved before it) into one constant per row, over the whole grid.  The
// segment's kernel then adds only in-segment terms: unknowns of the last W
// solve positions come from a shared-memory window (slot = position mod W),
// older ones from x through L2.  Each thread loads its records A levels
// before it needs them and, one level later, the older unknowns they read
// (finished by then), so the level-to-level critical path is the row's
// dependent FMAs on window values and the barrier.  Rows are stored divided
// by their diagonal: no division is left on that path.  On this GPU every
// FP64 instruction holds its pipe for many cycles, so a row's terms form one
// chain of FMAs (a second accumulator would cost an add and gain nothing
// with one warp per scheduler).

__global__ void tail_const_kernel(TailData td, const double *__restrict__ b,
                                  const double *__restrict__ x) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r = t >> 3;   // 8 lanes per row
    const int s = (int)(t & 7);
    double acc = 0.0;
    if (r < td.nrows) {
        const int64_t a = __ldg(&td.aptr[r]), e = __ldg(&td.aptr[r + 1]);
        for (int64_t k = a + s; k < e; k += 8) {
            const int32_t c = __ldg(&td.acol[k]);
            const double v = c >= 0 ? __ldcg(x + c) : __ldg(b + ~c);
            acc = fma(__ldg(&td.aval[k]), v, acc);
        }
    }
    acc += __shfl_xor_sync(FULL_MASK, acc, 4);
    acc += __shfl_xor_sync(FULL_MASK, acc, 2);
    acc += __shfl_xor_sync(FULL_MASK, acc, 1);
    if (r < td.nrows && s == 0) {
        const double br = __ldg(b + __ldg(&td.row[r]));
        const double2 dy = __ldg(&td.diag[r]);
        const bool scaled = (__ldg(&td.nn[r]) & kTailUnscaled) == 0;
        td.s0[r] = (scaled ? div_diag(br, dy.x, dy.y) : br) - acc;
    }
}

template <int K>
struct TailRec {
    int32_t row;   // -1: no row for this thread at this level
    int32_t pos, nn;
    double d, y, s0;
    int4 t[K];     // (slot or row, 0, value bits); once resolved, a far term holds
                   // (its unknown's bits, value bits)
};

// All loads unconditional on the record's own fields (no load waits on
// another), so issuing a prefetch never stalls the thread.
template <int K>
__device__ __forceinline__ void tail_load(const TailData &td, int32_t lo, int32_t hi,
                                          TailRec<K> &R) {
    const int32_t p = lo + (int32_t)threadIdx.x;
    R.row = -1;
    if (p < hi) {
        R.pos = p;
        R.row = __ldg(&td.row[p]);
        R.nn = __ldg(&td.nn[p]);
        const double2 dy = __ldg(&td.diag[p]);
        R.d = dy.x;
        R.y = dy.y;
        R.s0 = __ldcg(&td.s0[p]);
#pragma unroll
        for (int k = 0; k < K; ++k) R.t[k] = __ldg(&td.term[(int64_t)k * td.nrows + p]);
    }
}

// The far terms' unknowns (solved at least one level before the thread
// runs this), read from x into the record.
template <int K>
__device__ __forceinline__ void tail_resolve(const double *x, TailRec<K> &R) {
    if (R.row < 0) return;
    const int far = (R.nn >> 8) & 0xFFFF;
    if (!far) return;
#pragma unroll
    for (int k = 0; k < K; ++k)
        if (far & (1 << k)) {
            const long long v = __double_as_longlong(__ldcg(x + R.t[k].x));
            R.t[k].x = (int)(v & 0xFFFFFFFFll);
            R.t[k].y = (int)(v >> 32);
        }
}

__device__ __forceinline__ double lohi(int lo, int hi) {
    return __longlong_as_double(((long long)hi << 32) | (unsigned)lo);
}

template <int K>
__device__ __forceinline__ void tail_row(const TailData &td, const TailRec<K> &R,
                                         double *xs, double *x) {
    if (R.row < 0) return;
    const int cnt = R.nn & 0xFF, far = (R.nn >> 8) & 0xFFFF;
    // every window read issued at once (a far term's field holds value bits:
    // masked into the window, read and dropped), then one chain of FMAs
    double xv[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const double w = xs[R.t[k].x & (td.W - 1)];
        xv[k] = (far & (1 << k)) ? lohi(R.t[k].x, R.t[k].y) : w;
    }
    double acc = R.s0;
#pragma unroll
    for (int k = 0; k < K; ++k)
        if (k < cnt) acc = fma(-lohi(R.t[k].z, R.t[k].w), xv[k], acc);
    const double v = (R.nn & kTailUnscaled) ? div_diag(acc, R.d, R.y) : acc;
    xs[R.pos & (td.W - 1)] = v;
    x[R.row] = v;
}

template <int K, int A>
__global__ void __launch_bounds__(256, 1) tail_kernel(TailData td, double *__restrict__ x) {
    extern __shared__ double tail_xs[];
    for (int i = threadIdx.x; i < td.W; i += blockDim.x) tail_xs[i] = 0.0;
    const int32_t nl = td.nlev;
    TailRec<K> rec[A];
    int32_t blo[A], bhi[A];   // bounds of the level slot u loads next
#pragma unroll
    for (int u = 0; u < A; ++u) {
        if (u < nl) tail_load<K>(td, __ldg(&td.lp[u]), __ldg(&td.lp[u + 1]), rec[u]);
        else rec[u].row = -1;
        const int32_t l2 = u + A;
        blo[u] = l2 < nl ? __ldg(&td.lp[l2]) : 0;
        bhi[u] = l2 < nl ? __ldg(&td.lp[l2 + 1]) : 0;
    }
    __syncthreads();
    for (int32_t l0 = 0; l0 < nl; l0 += A) {
#pragma unroll
        for (int u = 0; u < A; ++u) {
            const int32_t l = l0 + u;
            if (l >= nl) break;   // uniform over the CTA
            tail_row<K>(td, rec[u], tail_xs, x);
            tail_load<K>(td, blo[u], bhi[u], rec[u]);   // level l + A
            // level l + A - 1, loaded one level ago: its far unknowns are
            // older than the window, so solved before level l, and have
            // A - 1 levels to arrive
            tail_resolve<K>(x, rec[(u + A - 1) % A]);
            const int32_t l2 = l + 2 * A;
            blo[u] = l2 < nl ? __ldg(&td.lp[l2]) : 0;
            bhi[u] = l2 < nl ? __ldg(&td.lp[l2 + 1]) : 0;
            __syncthreads();
        }
    }
}

}  // namespace

cudaError_t launch_tail_fold(const TailData &td, const double *b, const double *x,
                             cudaStream_t s) {
    if (td.nrows == 0) return cudaSuccess;
    const int64_t thr = (int64_t)td.nrows * 8;
    tail_const_kernel<<<(unsigned)((thr + 255) / 256), 256, 0, s>>>(td, b, x);
    return cudaGetLastError();
}

cudaError_t launch_tail(const TailData &td, const double *b, double *x, int block_threads,
                        cudaStream_t s) {
    if (td.nrows == 0 || td.nlev == 0) return cudaSuccess;
    if (block_threads < 32 || block_threads > 256 || (td.W & (td.W - 1)) != 0)
        return cudaErrorInvalidValue;
    cudaError_t e = launch_tail_fold(td, b, x, s);
    if (e != cudaSuccess) return e;
    const void *k = td.K <= 4   ? (const void *)tail_kernel<4, 4>
                    : td.K <= 8 ? (const void *)tail_kernel<8, 3>
                                : (const void *)tail_kernel<16, 2>;
    if (td.K > 16) return cudaErrorInvalidValue;
    const size_t smem = (size_t)td.W * sizeof(double);
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    TailData tc = td;
    void *args[] = {(void *)&tc, (void *)&x};
    return cudaLaunchKernel(k, dim3(1), dim3(block_threads), args, smem, s);
}

// The view of a segment the tail kernels take.
TailData tail_view(const TailSeg &t) {
    TailData d;
    d.nrows = t.nrows;
    d.nlev = t.nlev;
    d.K = t.K;
    d.W = t.W;
    d.lp = t.lp.p;
    d.row = t.row.p;
    d.nn = t.nn.p;
    d.term = t.term.p;
    d.diag = t.diag.p;
    d.aptr = t.aptr.p;
    d.acol = t.acol.p;
    d.aval = t.aval.p;
    d.s0 = t.s0.p;
    return d;
}

}  // namespace sptrsv
