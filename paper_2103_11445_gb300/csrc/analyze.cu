// Matrix analysis on the device (the paper's matrix-analysis module, Sec. IV):
// CSR validation, the level of every row of DAG_L (Sec. II) by a
// synchronisation-free pass in row order, and the level-ordered row
// permutation by a stable radix sort.
#include "kernels.cuh"

namespace sptrsv {
namespace {

// ---------------------------------------------------------------------------
// Validation: one thread per row.  row_ptr bounds are checked before any col
// entry of the row is read, so malformed pointers never cause a wild read.
// Error word: min over bad rows of (row << 8 | code): the first bad row wins.
__global__ void validate_kernel(int32_t n, int64_t nnz, const int32_t *__restrict__ row_ptr,
                                const int32_t *__restrict__ col,
                                const double *__restrict__ val,
                                int32_t *__restrict__ offdeg,
                                unsigned long long *err, unsigned long long *lnorm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int code = 0;
    const int64_t a = row_ptr[i], e = row_ptr[i + 1];
    if ((i == 0 && a != 0) || a < 0 || e < a || e > nnz || (i == n - 1 && e != nnz)) {
        code = SPTRSV_ERR_UNSORTED;
    } else if (a == e) {
        code = SPTRSV_ERR_MISSING_DIAG;
    } else {
        int64_t prev = -1;
        double rowabs = 0.0;
        for (int64_t k = a; k < e; ++k) {
            const int64_t c = col[k];
            if (c < 0 || c > i) { code = SPTRSV_ERR_NOT_LOWER; break; }
            if (c <= prev) { code = SPTRSV_ERR_UNSORTED; break; }
            prev = c;
            rowabs += fabs(val[k]);
        }
        if (!code) {
            if (col[e - 1] != i) code = SPTRSV_ERR_MISSING_DIAG;
            else if (val[e - 1] == 0.0) code = SPTRSV_ERR_ZERO_DIAG;
        }
        if (!code) {
            offdeg[i] = (int32_t)(e - a - 1);
            // non-negative doubles order like their bit patterns
            atomicMax(lnorm, (unsigned long long)__double_as_longlong(rowabs));
        }
    }
    if (code) atomicMin(err, ((unsigned long long)i << 8) | (unsigned long long)code);
}

// ---------------------------------------------------------------------------
// Level analysis without a barrier per level: level[i] = 0 for a row without
// dependencies, else 1 + the largest level among them (Sec. II), computed in
// row order by a persistent, co-resident grid.  Warp w takes rows w, w + nw,
// ... ; its lanes split the row's dependencies, poll (bounded) each one's
// level until it is set (levels start at -1) and reduce the maximum.  The
// lowest unfinished row's warp has finished its earlier rows and the row's
// dependencies all lie below it, so some warp can always make progress.
// The critical path is one poll hop per level instead of a grid barrier.
constexpr int kLevThreads = 256;

__device__ __forceinline__ int32_t ld_volatile_i32(const int32_t *p) {
    int32_t v;
    asm volatile("ld.volatile.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __noinline__ int32_t wait_level(const int32_t *p, DevStatus *st, uint64_t timeout_ns) {
    WaitBudget wb(timeout_ns);
    unsigned it = 0;
    int32_t v;
    do {
        if ((++it & kPollMask) == 0 && wb.expired(st, -6)) return -1;
        v = ld_volatile_i32(p);
    } while (v < 0);
    return v;
}

__global__ void __launch_bounds__(kLevThreads)
levels_syncfree_kernel(int32_t n, const int32_t *__restrict__ row_ptr,
                       const int32_t *__restrict__ col, int32_t *level, int32_t *nlev_out,
                       DevStatus *st, uint64_t timeout_ns) {
    const int lane = threadIdx.x & 31;
    const int32_t gw = (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int32_t nw = (int32_t)((gridDim.x * blockDim.x) >> 5);
    int32_t deepest = -1;
    for (int32_t i = gw; i < n; i += nw) {
        const int32_t a = __ldg(row_ptr + i), e = __ldg(row_ptr + i + 1) - 1;  // diagonal last
        int32_t m = -1;
        bool bail = false;
        for (int32_t k = a + lane; k < e; k += 32) {
            const int32_t *pj = level + __ldg(col + k);
            int32_t v = ld_volatile_i32(pj);
            if (v < 0) {
                v = wait_level(pj, st, timeout_ns);
                if (v < 0) bail = true;
            }
            m = max(m, v);
        }
        m = __reduce_max_sync(FULL_MASK, m);
        if (__any_sync(FULL_MASK, bail)) break;
        if (lane == 0) {
            asm volatile("st.volatile.global.b32 [%0], %1;" ::"l"(level + i), "r"(m + 1)
                         : "memory");
        }
        deepest = max(deepest, m + 1);
    }
    if (lane == 0 && deepest >= 0) atomicMax(nlev_out, deepest + 1);
}

// level_ptr[l] = first position of level l in perm (rows ordered by level);
// every level between 0 and the deepest holds a row, so each level starts
// where the level of the previous position changes.
__global__ void level_ptr_kernel(int32_t n, const int32_t *__restrict__ level,
                                 const int32_t *__restrict__ perm, int32_t nlev,
                                 int32_t *__restrict__ level_ptr) {
    const int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > n) return;
    const int32_t cur = p < n ? level[perm[p]] : nlev;
    const int32_t prev = p > 0 ? level[perm[p - 1]] : -1;
    for (int32_t l = prev + 1; l <= cur; ++l) level_ptr[l] = p;
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (key = level, value = row) pairs that start in row
// order; 8-bit digits.  Tiles of 2048 items: warp w of the block owns items
// [w*256, (w+1)*256) of the tile, visited in rounds of 32 consecutive items,
// so (warp, round, lane) order is the input order and per-warp ranks from
// __match_any_sync keep the sort stable.
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsRounds = 8;
constexpr int kRsTile = kRsThreads * kRsRounds;
constexpr int kRadix = 256;

__global__ void __launch_bounds__(kRsThreads)
radix_hist(const uint32_t *__restrict__ keys, int32_t n, int shift, int32_t *counts,
           int32_t nblocks) {
    __shared__ int32_t h[kRadix];
    for (int d = threadIdx.x; d < kRadix; d += kRsThreads) h[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int k = threadIdx.x; k < kRsTile; k += kRsThreads) {
        const int64_t idx = base + k;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & (kRadix - 1)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kRsThreads)
        counts[(int64_t)d * nblocks + blockIdx.x] = h[d];
}

__global__ void __launch_bounds__(kRsThreads)
radix_scatter(const uint32_t *__restrict__ keys_in, const int32_t *__restrict__ vals_in,
              uint32_t *__restrict__ keys_out, int32_t *__restrict__ vals_out,
              int32_t n, int shift, const int32_t *__restrict__ offsets,
              int32_t nblocks) {
    __shared__ int32_t wh[kRsWarps][kRadix];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < kRsWarps * kRadix; k += kRsThreads)
        (&wh[0][0])[k] = 0;
    __syncthreads();
    const int64_t wbase = (int64_t)blockIdx.x * kRsTile + warp * 32 * kRsRounds;
    // pass 1: per-warp digit counts
    for (int r = 0; r < kRsRounds; ++r) {
        const int64_t idx = wbase + r * 32 + lane;
        const bool valid = idx < n;
        const unsigned vmask = __ballot_sync(FULL_MASK, valid);
        if (valid) {
            const unsigned d = (keys_in[idx] >> shift) & (kRadix - 1);
            const unsigned peers = __match_any_sync(vmask, d);
            if (lane == __ffs(peers) - 1) wh[warp][d] += __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    // exclusive scan across warps, per digit
    for (int d = threadIdx.x; d < kRadix; d += kRsThreads) {
        int32_t run = offsets[(int64_t)d * nblocks + blockIdx.x];
        for (int w = 0; w < kRsWarps; ++w) {
            const int32_t t = wh[w][d];
            wh[w][d] = run;
            run += t;
        }
    }
    __syncthreads();
    // pass 2: stable scatter
    for (int r = 0; r < kRsRounds; ++r) {
        const int64_t idx = wbase + r * 32 + lane;
        const bool valid = idx < n;
        const unsigned vmask = __ballot_sync(FULL_MASK, valid);
        unsigned d = 0, peers = 0;
        int32_t pos = 0;
        if (valid) {
            const uint32_t key = keys_in[idx];
            d = (key >> shift) & (kRadix - 1);
            peers = __match_any_sync(vmask, d);
            pos = wh[warp][d] + __popc(peers & lanemask_lt());
            keys_out[pos] = key;
            vals_out[pos] = vals_in[idx];
        }
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wh[warp][d] += __popc(peers);
        __syncwarp();
    }
}

// rows by off-diagonal count: 0 | 1-2 | 3-6 | >= 7
__global__ void offdeg_hist_kernel(int32_t n, const int32_t *__restrict__ offdeg,
                                   unsigned long long *bins) {
    __shared__ unsigned long long h[4];
    if (threadIdx.x < 4) h[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = offdeg[i];
        atomicAdd(&h[d == 0 ? 0 : d <= 2 ? 1 : d <= 6 ? 2 : 3], 1ull);
    }
    __syncthreads();
    if (threadIdx.x < 4) atomicAdd(&bins[threadIdx.x], h[threadIdx.x]);
}

__global__ void iota_kernel(int32_t *v, int32_t n) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = i;
}

}  // namespace

cudaError_t launch_validate(int32_t n, int64_t nnz, const int32_t *row_ptr,
                            const int32_t *col, const double *val,
                            int32_t *offdeg, unsigned long long *err,
                            unsigned long long *lnorm, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    validate_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, nnz, row_ptr, col, val, offdeg,
                                                    err, lnorm);
    return cudaGetLastError();
}

cudaError_t launch_levels_syncfree(int32_t n, const int32_t *row_ptr, const int32_t *col,
                                   int32_t *level, int32_t *nlev_out, DevStatus *st,
                                   uint64_t timeout_ns, int num_sms, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, levels_syncfree_kernel, kLevThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    int64_t grid = (int64_t)per_sm * num_sms;
    const int64_t want = ((int64_t)n * 32 + kLevThreads - 1) / kLevThreads;
    if (want < grid) grid = want;
    if ((e = cudaMemsetAsync(level, 0xff, (size_t)n * sizeof(int32_t), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(nlev_out, 0, sizeof(int32_t), s)) != cudaSuccess) return e;
    void *args[] = {(void *)&n, (void *)&row_ptr, (void *)&col, (void *)&level,
                    (void *)&nlev_out, (void *)&st, (void *)&timeout_ns};
    return cudaLaunchCooperativeKernel((void *)levels_syncfree_kernel, dim3((unsigned)grid),
                                       dim3(kLevThreads), args, 0, s);
}

cudaError_t launch_level_ptr(int32_t n, const int32_t *level, const int32_t *perm, int32_t nlev,
                             int32_t *level_ptr, cudaStream_t s) {
    level_ptr_kernel<<<(unsigned)(((int64_t)n + 256) / 256), 256, 0, s>>>(n, level, perm, nlev,
                                                                        level_ptr);
    return cudaGetLastError();
}

cudaError_t launch_offdeg_hist(int32_t n, const int32_t *offdeg, unsigned long long *bins,
                               cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    int64_t blocks = ((int64_t)n + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    offdeg_hist_kernel<<<(unsigned)blocks, 256, 0, s>>>(n, offdeg, bins);
    return cudaGetLastError();
}

size_t radix_tmp_bytes(int32_t n) {
    const int64_t nb = ((int64_t)n + kRsTile - 1) / kRsTile;
    const int64_t cnt = (int64_t)kRadix * (nb > 0 ? nb : 1);
    size_t b = 0;
    b += 2 * (size_t)n * sizeof(uint32_t);       // keys ping-pong
    b += (size_t)n * sizeof(int32_t);            // values ping (pong = perm)
    b += (size_t)(cnt + 1) * sizeof(int32_t);    // counts -> offsets
    b += (size_t)scan_tmp_elems(cnt) * sizeof(int64_t);
    return b + 256 * 6;
}

cudaError_t launch_level_perm(int32_t n, const int32_t *level, int32_t nlev,
                              int32_t *perm, void *tmp, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int32_t nb = (int32_t)(((int64_t)n + kRsTile - 1) / kRsTile);
    const int64_t cnt = (int64_t)kRadix * nb;
    auto align = [](char *p) { return (char *)(((uintptr_t)p + 255) & ~(uintptr_t)255); };
    char *p = align((char *)tmp);
    uint32_t *ka = (uint32_t *)p;  p = align(p + (size_t)n * 4);
    uint32_t *kb = (uint32_t *)p;  p = align(p + (size_t)n * 4);
    int32_t *va = (int32_t *)p;    p = align(p + (size_t)n * 4);
    int32_t *counts = (int32_t *)p; p = align(p + (size_t)(cnt + 1) * 4);
    int64_t *stmp = (int64_t *)p;
    int passes = 1;
    while (passes < 4 && ((uint64_t)(nlev > 0 ? nlev - 1 : 0) >> (8 * passes)) != 0) ++passes;
    // keys = level (copied so the plan's level array stays untouched)
    cudaError_t e = cudaMemcpyAsync(ka, level, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    // values: start in row order, finish in perm
    int32_t *v_in = (passes % 2 == 0) ? perm : va;
    int32_t *v_out = (passes % 2 == 0) ? va : perm;
    iota_kernel<<<(n + 255) / 256, 256, 0, s>>>(v_in, n);
    uint32_t *k_in = ka, *k_out = kb;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        radix_hist<<<nb, kRsThreads, 0, s>>>(k_in, n, shift, counts, nb);
        e = exclusive_scan_i32_i32(counts, counts, cnt, stmp, s);
        if (e != cudaSuccess) return e;
        radix_scatter<<<nb, kRsThreads, 0, s>>>(k_in, v_in, k_out, v_out, n, shift, counts, nb);
        std::swap(k_in, k_out);
        std::swap(v_in, v_out);
    }
    return cudaGetLastError();
}

}  // namespace sptrsv
