// Matrix analysis on the device (the paper's matrix-analysis module, Sec. IV):
// CSR validation, the successor lists of DAG_L (Sec. II), the level of every
// row by a breadth-first (Kahn) traversal of DAG_L, and the level-ordered
// row permutation by a stable radix sort.
#include <cooperative_groups.h>

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

__global__ void count_succ_kernel(int32_t n, const int32_t *__restrict__ row_ptr,
                                  const int32_t *__restrict__ col, int32_t *tcnt) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t k = row_ptr[i]; k < row_ptr[i + 1] - 1; ++k) atomicAdd(&tcnt[col[k]], 1);
}

__global__ void fill_succ_kernel(int32_t n, const int32_t *__restrict__ row_ptr,
                                 const int32_t *__restrict__ col,
                                 const int32_t *__restrict__ tptr, int32_t *tcur,
                                 int32_t *tidx) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t k = row_ptr[i]; k < row_ptr[i + 1] - 1; ++k) {
        const int32_t j = col[k];
        tidx[tptr[j] + atomicAdd(&tcur[j], 1)] = i;
    }
}

// ---------------------------------------------------------------------------
// Breadth-first level analysis in one cooperative launch.  Round m expands
// the frontier of level m (queue[lo, hi)): every successor whose remaining
// in-degree drops to zero joins level m+1 and is appended behind hi through
// counter cnt3[(m+1) % 3].  After the grid barrier every CTA reads that
// counter to learn the next frontier.  Three counters rotate so that a
// counter is reset (during round m, for use in round m+2... i.e. the one
// last read before the previous barrier) while nobody reads or appends it.
constexpr int kBfsThreads = 512;

__global__ void __launch_bounds__(kBfsThreads)
bfs_levels_kernel(int32_t n, const int32_t *__restrict__ tptr,
                  const int32_t *__restrict__ tidx, int32_t *indeg, int32_t *level,
                  int32_t *queue, int32_t *cnt3, int32_t *level_start,
                  int32_t *nlev_out, DevStatus *st, uint64_t timeout_ns) {
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
    unsigned long long bar = 0;
    // level 0: rows without dependencies
    for (int64_t i = gtid; i < n; i += gthreads) {
        if (indeg[i] == 0) {
            level[i] = 0;
            queue[atomicAdd(&cnt3[0], 1)] = (int32_t)i;
        }
    }
    bool ok = grid_barrier(st, (++bar) * gridDim.x, timeout_ns, -1);
    int32_t lo = 0;
    int32_t hi = ok ? (int32_t)ld_relaxed_u32(&cnt3[0]) : 0;
    int32_t m = 0;
    while (ok && hi > lo) {
        if (gtid == 0) {
            level_start[m] = lo;
            cnt3[(m + 2) % 3] = 0;  // last read before the previous barrier
        }
        int32_t *next_cnt = &cnt3[(m + 1) % 3];
        for (int64_t q = lo + gtid; q < hi; q += gthreads) {
            const int32_t r = __ldcg(&queue[q]);
            const int32_t e = tptr[r + 1];
            for (int32_t k = tptr[r]; k < e; ++k) {
                const int32_t s = tidx[k];
                if (atomicSub(&indeg[s], 1) == 1) {
                    level[s] = m + 1;
                    queue[hi + atomicAdd(next_cnt, 1)] = s;
                }
            }
        }
        ok = grid_barrier(st, (++bar) * gridDim.x, timeout_ns, m);
        const int32_t sz = ok ? (int32_t)ld_relaxed_u32(next_cnt) : 0;
        lo = hi;
        hi += sz;
        ++m;
    }
    if (gtid == 0) {
        level_start[m] = lo;
        *nlev_out = ok ? m : -1;
    }
    grid_exit(st);
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

cudaError_t launch_count_succ(int32_t n, const int32_t *row_ptr, const int32_t *col,
                              int32_t *tcnt, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    count_succ_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, row_ptr, col, tcnt);
    return cudaGetLastError();
}

cudaError_t launch_fill_succ(int32_t n, const int32_t *row_ptr, const int32_t *col,
                             const int32_t *tptr, int32_t *tcur, int32_t *tidx,
                             cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    fill_succ_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, row_ptr, col, tptr, tcur, tidx);
    return cudaGetLastError();
}

cudaError_t launch_bfs_levels(int32_t n, const int32_t *tptr, const int32_t *tidx,
                              int32_t *indeg, int32_t *level, int32_t *queue,
                              int32_t *cnt3, int32_t *level_start,
                              int32_t *nlev_out, DevStatus *st,
                              uint64_t timeout_ns, int num_sms, cudaStream_t s) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, bfs_levels_kernel, kBfsThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    // one CTA per SM keeps the barrier cheap; the frontier loop is grid-strided
    int grid = num_sms;
    int64_t want = ((int64_t)n + kBfsThreads - 1) / kBfsThreads;
    if (want < grid) grid = (int)(want > 0 ? want : 1);
    void *args[] = {(void *)&n, (void *)&tptr, (void *)&tidx, (void *)&indeg,
                    (void *)&level, (void *)&queue, (void *)&cnt3, (void *)&level_start,
                    (void *)&nlev_out, (void *)&st, (void *)&timeout_ns};
    return cudaLaunchCooperativeKernel((void *)bfs_levels_kernel, dim3(grid),
                                       dim3(kBfsThreads), args, 0, s);
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
