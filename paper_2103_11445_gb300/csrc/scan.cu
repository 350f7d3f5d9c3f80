// Device-wide exclusive prefix sums (reduce, scan of tile sums, scan tiles).
// Used for CSR-style offsets everywhere in the analysis and the transform.
#include "kernels.cuh"

namespace sptrsv {
namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// Exclusive scan of one value per thread across the block; returns the
// prefix and writes the block total to *total.
__device__ __forceinline__ int64_t block_exclusive(int64_t v, int64_t *total) {
    constexpr int NW = kScanThreads / 32;
    __shared__ int64_t warp_sums[NW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(FULL_MASK, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < NW ? warp_sums[lane] : 0;
        int64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(FULL_MASK, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < NW) warp_sums[lane] = wi - w;
        if (lane == NW - 1) *total = wi;
    }
    __syncthreads();
    int64_t r = warp_sums[warp] + inc - v;
    __syncthreads();  // warp_sums and *total may be reused by the next call
    return r;
}

template <typename Tin>
__global__ void __launch_bounds__(kScanThreads)
tile_reduce(const Tin *in, int64_t n, int64_t *bsum) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += (int64_t)in[base + k];
    __shared__ int64_t tot;
    block_exclusive(s, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// single block: exclusive scan of nb tile sums in place, grand total in *total
__global__ void __launch_bounds__(kScanThreads)
scan_tile_sums(int64_t *bsum, int64_t nb, int64_t *total) {
    __shared__ int64_t carry_s, tot;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += kScanTile) {
        int64_t idx = base + (int64_t)threadIdx.x * kScanItems;
        int64_t v[kScanItems];
        int64_t s = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            v[k] = idx + k < nb ? bsum[idx + k] : 0;
            s += v[k];
        }
        int64_t pre = block_exclusive(s, &tot) + carry_s;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (idx + k < nb) bsum[idx + k] = pre;
            pre += v[k];
        }
        __syncthreads();
        if (threadIdx.x == 0) carry_s += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry_s;
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kScanThreads)
tile_scan(const Tin *in, Tout *out, int64_t n, const int64_t *bsum,
          const int64_t *total) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? (int64_t)in[base + k] : 0;
        s += v[k];
    }
    __shared__ int64_t tot;
    int64_t pre = block_exclusive(s, &tot) + bsum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = (Tout)pre;
        pre += v[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = (Tout)*total;
}

template <typename Tin, typename Tout>
cudaError_t scan_impl(const Tin *in, Tout *out, int64_t n, int64_t *tmp, cudaStream_t s) {
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    int64_t *bsum = tmp, *total = tmp + (nb > 0 ? nb : 1);
    if (nb == 0) {
        // empty input: out[0] = 0
        cudaError_t e = cudaMemsetAsync(total, 0, sizeof(int64_t), s);
        if (e != cudaSuccess) return e;
        tile_scan<Tin, Tout><<<1, kScanThreads, 0, s>>>(in, out, 0, total, total);
        return cudaGetLastError();
    }
    tile_reduce<Tin><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, bsum);
    scan_tile_sums<<<1, kScanThreads, 0, s>>>(bsum, nb, total);
    tile_scan<Tin, Tout><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, bsum, total);
    return cudaGetLastError();
}

}  // namespace

int64_t scan_tmp_elems(int64_t n) { return (n + kScanTile - 1) / kScanTile + 2; }

cudaError_t exclusive_scan_i32_i64(const int32_t *in, int64_t *out, int64_t n,
                                   int64_t *tmp, cudaStream_t s) {
    return scan_impl<int32_t, int64_t>(in, out, n, tmp, s);
}
cudaError_t exclusive_scan_i64_i64(const int64_t *in, int64_t *out, int64_t n,
                                   int64_t *tmp, cudaStream_t s) {
    return scan_impl<int64_t, int64_t>(in, out, n, tmp, s);
}
cudaError_t exclusive_scan_i32_i32(const int32_t *in, int32_t *out, int64_t n,
                                   int64_t *tmp, cudaStream_t s) {
    return scan_impl<int32_t, int32_t>(in, out, n, tmp, s);
}

}  // namespace sptrsv
