// Equation rewriting on the device (Sec. III, Figs. 2-3) and assembly of the
// level-ordered solve structure.
//
// A rewritten row i with target level t is the row operation
//     row_i  <-  row_i - sum_{j in S} c_j row_j
// where S holds every dependency reachable from i through rows of level >= t.
// It is computed by substituting original equations, always the largest
// remaining dependency of level >= t first (Fig. 2 substitutes row 1, then
// row 0): m = coef[j] / L_jj, coef[k] -= m L_jk for the entries of row j,
// c_j = m.  New dependencies are always smaller than j, so one descending
// sweep over a sorted pattern visits each j once.  The right-hand side of the
// rearranged row (Fig. 3) is b_i - sum c_j b_j, applied at solve time.
//
// One warp per rewritten row keeps the row's pattern sorted in shared
// memory: a double-buffered sorted array merged with the new entries of each
// substituted row.  FP64 throughout (cancellation happens here).
#include "transform.cuh"

namespace sptrsv {
namespace {

__device__ __forceinline__ int lower_bound_smem(const int32_t *a, int lo, int hi, int32_t v) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Per-warp workspace: A (current pattern), B (merge target), N (new entries).
struct WarpWs {
    int32_t *ac, *bc, *nc;
    double *av, *bv, *nv;
};

template <bool NUMERIC>
__device__ int rewrite_one(int32_t row, int32_t t, const int32_t *__restrict__ row_ptr,
                           const int32_t *__restrict__ col, const double *__restrict__ val,
                           const int32_t *__restrict__ level, int cap, WarpWs ws) {
    const int lane = threadIdx.x & 31;
    const int32_t a = row_ptr[row];
    int m = row_ptr[row + 1] - 1 - a;
    if (m > cap) return -1;
    int32_t *ac = ws.ac, *bc = ws.bc;
    double *av = ws.av, *bv = ws.bv;
    for (int k = lane; k < m; k += 32) {
        ac[k] = col[a + k];
        if (NUMERIC) av[k] = val[a + k];
    }
    __syncwarp();
    int q = m;
    while (true) {
        // highest index below q whose column lies at level >= t
        int idx = -1;
        for (int base = q - 1; base >= 0; base -= 32) {
            const int k = base - lane;
            const bool f = k >= 0 && level[ac[k]] >= t;
            const unsigned bal = __ballot_sync(FULL_MASK, f);
            if (bal) { idx = base - (__ffs(bal) - 1); break; }
        }
        if (idx < 0) break;
        const int32_t j = ac[idx];
        double mj = 0.0;
        if (NUMERIC) mj = av[idx] / val[row_ptr[j + 1] - 1];
        __syncwarp();
        if (NUMERIC && lane == 0) av[idx] = mj;  // the entry now holds c_j
        __syncwarp();
        // entries of row j: update present ones, collect new ones (sorted)
        const int32_t ja = row_ptr[j], je = row_ptr[j + 1] - 1;
        int nnew = 0;
        for (int32_t cb = ja; cb < je; cb += 32) {
            const int32_t k = cb + lane;
            const bool valid = k < je;
            const int32_t c = valid ? col[k] : 0;
            const double v = (NUMERIC && valid) ? val[k] : 0.0;
            const int pos = valid ? lower_bound_smem(ac, 0, idx, c) : 0;
            const bool present = valid && pos < idx && ac[pos] == c;
            if (NUMERIC && present) av[pos] -= mj * v;
            const bool isnew = valid && !present;
            const unsigned bal = __ballot_sync(FULL_MASK, isnew);
            const int cnt = __popc(bal);
            if (m + nnew + cnt > cap) return -1;
            if (isnew) {
                const int r = nnew + __popc(bal & lanemask_lt());
                ws.nc[r] = c;
                if (NUMERIC) ws.nv[r] = -mj * v;
            }
            nnew += cnt;
        }
        __syncwarp();
        if (nnew > 0) {
            for (int k = lane; k < idx; k += 32) {
                const int32_t c = ac[k];
                const int d = k + lower_bound_smem(ws.nc, 0, nnew, c);
                bc[d] = c;
                if (NUMERIC) bv[d] = av[k];
            }
            for (int k = lane; k < nnew; k += 32) {
                const int32_t c = ws.nc[k];
                const int d = k + lower_bound_smem(ac, 0, idx, c);
                bc[d] = c;
                if (NUMERIC) bv[d] = ws.nv[k];
            }
            for (int k = idx + lane; k < m; k += 32) {
                bc[k + nnew] = ac[k];
                if (NUMERIC) bv[k + nnew] = av[k];
            }
            __syncwarp();
            int32_t *tc = ac; ac = bc; bc = tc;
            double *tv = av; av = bv; bv = tv;
            m += nnew;
        }
        q = idx + nnew;
    }
    // the final pattern lives in (ac, av); hand it back through ws.ac/av
    if (ac != ws.ac) {
        for (int k = lane; k < m; k += 32) {
            ws.ac[k] = ac[k];
            if (NUMERIC) ws.av[k] = av[k];
        }
    }
    __syncwarp();
    return m;
}

__device__ __forceinline__ WarpWs carve(char *smem, int warp, int cap, bool numeric) {
    const size_t per = (size_t)cap * (numeric ? 3 * (4 + 8) : 3 * 4) + 16;
    char *p = smem + per * warp;
    WarpWs ws;
    ws.ac = (int32_t *)p;
    ws.bc = ws.ac + cap;
    ws.nc = ws.bc + cap;
    if (numeric) {
        double *v = (double *)(((uintptr_t)(ws.nc + cap) + 7) & ~(uintptr_t)7);
        ws.av = v;
        ws.bv = v + cap;
        ws.nv = v + 2 * cap;
    } else {
        ws.av = ws.bv = ws.nv = nullptr;
    }
    return ws;
}

// Count mode: fill of each (row, target) item; per query q adds
// 2 * (fill - offdeg) to added[q] or flags an overflow.
__global__ void rewrite_count_kernel(int64_t nitems, const int32_t *__restrict__ item_row,
                                     const int32_t *__restrict__ item_tgt,
                                     const int32_t *__restrict__ item_q,
                                     const int32_t *__restrict__ row_ptr,
                                     const int32_t *__restrict__ col,
                                     const int32_t *__restrict__ level, int cap,
                                     int32_t *fill_out, unsigned long long *added,
                                     int32_t *overflow, int32_t *maxlen) {
    extern __shared__ __align__(16) char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    WarpWs ws = carve(smem, warp, cap, false);
    for (int64_t it = (int64_t)blockIdx.x * wpb + warp; it < nitems;
         it += (int64_t)gridDim.x * wpb) {
        const int32_t row = item_row[it];
        const int f = rewrite_one<false>(row, item_tgt[it], row_ptr, col, nullptr, level,
                                         cap, ws);
        if (lane == 0) {
            if (fill_out) fill_out[it] = f;
            if (item_q) {
                const int32_t q = item_q[it];
                if (f < 0) {
                    atomicExch(&overflow[q], 1);
                } else {
                    atomicAdd(&added[q], (unsigned long long)(2ll * (f - (row_ptr[row + 1] - 1 - row_ptr[row]))));
                    if (maxlen) atomicMax(&maxlen[q], f);
                }
            }
        }
        __syncwarp();
    }
}

// Numeric mode: writes item it's entries at out_off[it]: first the
// eliminated set S (encoded ~j, weight c_j), then the x terms (col, coef),
// each ascending.  nb_out[it] = |S|.
__global__ void rewrite_numeric_kernel(int64_t nitems, const int32_t *__restrict__ item_row,
                                       const int32_t *__restrict__ item_tgt,
                                       const int64_t *__restrict__ out_off,
                                       const int32_t *__restrict__ row_ptr,
                                       const int32_t *__restrict__ col,
                                       const double *__restrict__ val,
                                       const int32_t *__restrict__ level, int cap,
                                       int32_t *out_col, double *out_val, int32_t *nb_out,
                                       DevStatus *st) {
    extern __shared__ __align__(16) char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    WarpWs ws = carve(smem, warp, cap, true);
    for (int64_t it = (int64_t)blockIdx.x * wpb + warp; it < nitems;
         it += (int64_t)gridDim.x * wpb) {
        const int32_t t = item_tgt[it];
        const int m = rewrite_one<true>(item_row[it], t, row_ptr, col, val, level, cap, ws);
        const int64_t base = out_off[it];
        if (m < 0 || m != out_off[it + 1] - base) {
            if (lane == 0) latch_error(st, SPTRSV_ERR_BAD_STATE, (int)it);
            continue;
        }
        // partition: S (level >= t) first, then x terms, both ascending
        int ns_total = 0;
        for (int k0 = 0; k0 < m; k0 += 32) {
            const int k = k0 + lane;
            const bool in = k < m && level[ws.ac[k]] >= t;
            ns_total += __popc(__ballot_sync(FULL_MASK, in));
        }
        int ns = 0, nx = 0;
        for (int k0 = 0; k0 < m; k0 += 32) {
            const int k = k0 + lane;
            const bool valid = k < m;
            const int32_t c = valid ? ws.ac[k] : 0;
            const bool inS = valid && level[c] >= t;
            const unsigned bs = __ballot_sync(FULL_MASK, inS);
            const unsigned bx = __ballot_sync(FULL_MASK, valid && !inS);
            if (inS) {
                const int64_t d = base + ns + __popc(bs & lanemask_lt());
                out_col[d] = ~c;
                out_val[d] = ws.av[k];
            } else if (valid) {
                const int64_t d = base + ns_total + nx + __popc(bx & lanemask_lt());
                out_col[d] = c;
                out_val[d] = ws.av[k];
            }
            ns += __popc(bs);
            nx += __popc(bx);
        }
        if (lane == 0) nb_out[it] = ns_total;
        __syncwarp();
    }
}

// items of a list of (level, target) queries: rows perm[level_ptr[l] ..)
__global__ void expand_queries_kernel(int32_t nq, const int32_t *__restrict__ q_level,
                                      const int32_t *__restrict__ q_tgt,
                                      const int64_t *__restrict__ q_off,
                                      const int32_t *__restrict__ level_ptr,
                                      const int32_t *__restrict__ perm,
                                      int32_t *item_row, int32_t *item_tgt, int32_t *item_q,
                                      int32_t *item_pos) {
    const int32_t q = blockIdx.x;
    if (q >= nq) return;
    const int32_t l = q_level[q];
    const int32_t p0 = level_ptr[l], p1 = level_ptr[l + 1];
    const int64_t o = q_off[q];
    for (int32_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        const int64_t it = o + (p - p0);
        item_row[it] = perm[p];
        item_tgt[it] = q_tgt[q];
        if (item_q) item_q[it] = q;
        if (item_pos) item_pos[it] = p;
    }
}

__global__ void scatter_item_index(int64_t nitems, const int32_t *__restrict__ item_pos,
                                   int32_t *pos_item) {
    const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it < nitems) pos_item[item_pos[it]] = (int32_t)it;
}

__global__ void fill_i32(int32_t *p, int64_t n, int32_t v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// ---------------------------------------------------------------------------
// Assembly of the solve structure.

__device__ __forceinline__ int32_t pos_len(int32_t p, const int32_t *perm,
                                           const int32_t *offdeg, const int32_t *pos_item,
                                           const int64_t *rw_off) {
    const int32_t it = pos_item ? pos_item[p] : -1;
    if (it >= 0) return (int32_t)(rw_off[it + 1] - rw_off[it]);
    return offdeg[perm[p]];
}

__global__ void chunk_width_kernel(int32_t nchunks, const int32_t *__restrict__ c_row0,
                                   const int32_t *__restrict__ c_nrows, int L,
                                   const int32_t *__restrict__ perm,
                                   const int32_t *__restrict__ offdeg,
                                   const int32_t *__restrict__ pos_item,
                                   const int64_t *__restrict__ rw_off,
                                   int64_t *slots, int32_t *width_out) {
    const int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nchunks) return;
    const int32_t r0 = c_row0[c], nr = c_nrows[c];
    int32_t w = 0;
    for (int32_t k = 0; k < nr; ++k) {
        const int32_t len = pos_len(r0 + k, perm, offdeg, pos_item, rw_off);
        const int32_t s = (len + L - 1) / L;
        w = s > w ? s : w;
    }
    width_out[c] = w;
    // a multiple of 4 entries: chunks start on 16-byte boundaries
    slots[c] = ((int64_t)w * nr * L + 3) & ~(int64_t)3;
}

// one thread per (chunk, row-in-chunk): writes the row's entries and pads
template <typename T>
__global__ void chunk_fill_kernel(int32_t nchunks, int H, int L,
                                  const int32_t *__restrict__ c_row0,
                                  const int32_t *__restrict__ c_nrows,
                                  const int32_t *__restrict__ c_width,
                                  const int64_t *__restrict__ c_off,
                                  const int32_t *__restrict__ perm,
                                  const int32_t *__restrict__ row_ptr,
                                  const int32_t *__restrict__ col,
                                  const double *__restrict__ val,
                                  const int32_t *__restrict__ pos_item,
                                  const int64_t *__restrict__ rw_off,
                                  const int32_t *__restrict__ rw_col,
                                  const double *__restrict__ rw_val,
                                  int4 *meta, int32_t *ecol, T *eval, int32_t *row_id,
                                  T *diag) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t c = g / H;
    const int k = (int)(g % H);
    if (c >= nchunks) return;
    const int32_t nr = c_nrows[c];
    const int32_t w = c_width[c];
    const int64_t off = c_off[c];
    if (k == 0) meta[c] = make_int4(c_row0[c], nr, w, (int32_t)off);
    if (k >= nr) return;
    const int32_t p = c_row0[c] + k;
    const int32_t r = perm[p];
    row_id[p] = r;
    const int32_t dpos = row_ptr[r + 1] - 1;
    // (L_ii, RN(1/L_ii)); the reciprocal is 0 where the solve must divide
    const T d = (T)val[dpos];
    const T ad = fabs(d);
    const bool safe = sizeof(T) == 8 ? (ad >= (T)0x1p-1000 && ad <= (T)0x1p+1000)
                                     : (ad >= (T)0x1p-120f && ad <= (T)0x1p+120f);
    diag[2 * (int64_t)p] = d;
    diag[2 * (int64_t)p + 1] = safe ? T(1) / d : T(0);
    const int32_t it = pos_item ? pos_item[p] : -1;
    const int64_t stride = (int64_t)nr * L;
    int32_t len;
    const int32_t *src_c;
    const double *src_v;
    if (it >= 0) {
        len = (int32_t)(rw_off[it + 1] - rw_off[it]);
        src_c = rw_col + rw_off[it];
        src_v = rw_val + rw_off[it];
    } else {
        len = dpos - row_ptr[r];
        src_c = col + row_ptr[r];
        src_v = val + row_ptr[r];
    }
    const int32_t total = w * L;
    for (int32_t j = 0; j < total; ++j) {
        const int64_t slot = off + (int64_t)(j / L) * stride + (int64_t)k * L + (j % L);
        if (j < len) {
            ecol[slot] = src_c[j];
            eval[slot] = (T)src_v[j];
        } else {
            ecol[slot] = PAD_COL;
            eval[slot] = (T)0;
        }
    }
}

// Export (tests): per original row, counts of x and b terms.  Columns
// < -n (not PAD) are run slots of a CTA-local run: x terms.
__global__ void export_count_kernel(int32_t nchunks, int H, int L, const int4 *__restrict__ meta,
                                    const int32_t *__restrict__ ecol,
                                    const int32_t *__restrict__ row_id, int32_t n,
                                    int64_t *xcnt, int64_t *bcnt) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t c = g / H;
    const int k = (int)(g % H);
    if (c >= nchunks) return;
    const int4 mt = meta[c];
    if (k >= mt.y) return;
    const int64_t stride = (int64_t)mt.y * L;
    int64_t nx = 0, nb = 0;
    for (int32_t j = 0; j < mt.z * L; ++j) {
        const int32_t cc = ecol[mt.w + (int64_t)(j / L) * stride + (int64_t)k * L + (j % L)];
        if (cc == PAD_COL) continue;
        if (cc >= 0 || cc < -n) ++nx; else ++nb;
    }
    const int32_t r = row_id[mt.x + k];
    xcnt[r] = nx;
    bcnt[r] = nb;
}

template <typename T>
__global__ void export_fill_kernel(int32_t nchunks, int H, int L, const int4 *__restrict__ meta,
                                   const int32_t *__restrict__ ecol, const T *__restrict__ eval,
                                   const int32_t *__restrict__ row_id,
                                   const int32_t *__restrict__ chunk_level,
                                   const int32_t *__restrict__ chunk_run_p0, int32_t n,
                                   const int64_t *__restrict__ xptr,
                                   const int64_t *__restrict__ bptr, int32_t *xcol,
                                   double *xval, int32_t *bcol, double *bw,
                                   int32_t *new_level) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t c = g / H;
    const int k = (int)(g % H);
    if (c >= nchunks) return;
    const int4 mt = meta[c];
    if (k >= mt.y) return;
    const int64_t stride = (int64_t)mt.y * L;
    const int32_t r = row_id[mt.x + k];
    int64_t px = xptr ? xptr[r] : 0, pb = bptr ? bptr[r] : 0;
    for (int32_t j = 0; j < mt.z * L; ++j) {
        const int64_t slot = mt.w + (int64_t)(j / L) * stride + (int64_t)k * L + (j % L);
        int32_t cc = ecol[slot];
        if (cc == PAD_COL) continue;
        if (cc < -n) cc = row_id[chunk_run_p0[c] + (-(n + 1) - cc)];  // run slot -> row
        if (cc >= 0) {
            if (xcol) xcol[px] = cc;
            if (xval) xval[px] = (double)eval[slot];
            ++px;
        } else {
            if (bcol) bcol[pb] = ~cc;
            if (bw) bw[pb] = (double)eval[slot];
            ++pb;
        }
    }
    if (new_level) new_level[r] = chunk_level[c];
}

__global__ void chunk_level_kernel(int32_t nlev, const int32_t *__restrict__ lvl_chunk,
                                   int32_t *chunk_level) {
    const int32_t l = blockIdx.x;
    if (l >= nlev) return;
    for (int32_t c = lvl_chunk[l] + threadIdx.x; c < lvl_chunk[l + 1]; c += blockDim.x)
        chunk_level[c] = l;
}

__global__ void pos_of_row_kernel(int32_t n, const int32_t *__restrict__ row_id,
                                  int32_t *__restrict__ pos) {
    const int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) pos[row_id[p]] = p;
}

// Run chunks: an x term whose row lies in the same run [P0, P1) of solve
// positions becomes the shared-memory slot -(n + 1) - (pos - P0).
__global__ void encode_run_kernel(int32_t nrc, const int32_t *__restrict__ run_chunk,
                                  const int2 *__restrict__ run_span, int H, int L, int32_t n,
                                  const int4 *__restrict__ meta, const int32_t *__restrict__ pos,
                                  int32_t *__restrict__ ecol) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = g / H;
    const int k = (int)(g % H);
    if (i >= nrc) return;
    const int4 mt = meta[run_chunk[i]];
    if (k >= mt.y) return;
    const int2 span = run_span[i];
    const int64_t stride = (int64_t)mt.y * L;
    for (int32_t j = 0; j < mt.z * L; ++j) {
        const int64_t slot = mt.w + (int64_t)(j / L) * stride + (int64_t)k * L + (j % L);
        const int32_t c = ecol[slot];
        if (c < 0) continue;
        const int32_t q = pos[c];
        if (q >= span.x && q < span.y) ecol[slot] = -(n + 1) - (q - span.x);
    }
}

__global__ void f64_to_f32(const double *__restrict__ a, float *__restrict__ b, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

int warps_for_cap(int cap, bool numeric, size_t *smem) {
    const size_t per = (size_t)cap * (numeric ? 3 * (4 + 8) : 3 * 4) + 16;
    int w = (int)((200 * 1024) / per);
    if (w > 8) w = 8;
    if (w < 1) w = 1;
    *smem = per * w + 16;
    return w;
}


// ---- single-CTA tail: records built from the solve structure --------------

// One thread per tail chunk: per row, the terms folded into the constant
// (b terms, unknowns before the tail) and the in-tail terms; the largest
// in-tail count goes to *kmax.  A run-slot entry (never present in a
// structure built for the tail) sets *bad.
__global__ void tail_count_kernel(int32_t c0, int32_t nchunks, int L, int32_t n,
                                  const int4 *__restrict__ meta, const int32_t *__restrict__ ecol,
                                  const int32_t *__restrict__ pos_of, int32_t P0,
                                  int32_t *__restrict__ cnt_a, int32_t *__restrict__ cnt_n,
                                  int32_t *kmax, int32_t *bad) {
    const int32_t c = c0 + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (c >= nchunks) return;
    const int4 mt = meta[c];
    const int64_t stride = (int64_t)mt.y * L;
    for (int32_t k = 0; k < mt.y; ++k) {
        int32_t na = 0, nn = 0;
        for (int32_t t = 0; t < mt.z; ++t)
            for (int sl = 0; sl < L; ++sl) {
                const int32_t col = ecol[mt.w + t * stride + (int64_t)k * L + sl];
                if (col == PAD_COL) continue;
                if (col >= 0) {
                    if (pos_of[col] >= P0) ++nn;
                    else ++na;
                } else if (col >= -n) {
                    ++na;
                } else {
                    *bad = 1;
                }
            }
        cnt_a[mt.x + k - P0] = na;
        cnt_n[mt.x + k - P0] = nn;
        atomicMax(kmax, nn);
    }
}

// The records: a term of row p reading tail position q is near when
// (start of p's level) - q <= W - T (its window slot is not overwritten
// before p's level), far (read from x; bit k of the row's far mask) otherwise.
// A row's coefficients -- in-tail terms and folded ones -- are stored divided
// by its diagonal (IEEE division), unless the quotient of a non-zero
// coefficient leaves the normal range: then the row keeps them as they are
// and is marked kTailUnscaled.
__global__ void tail_fill_kernel(int32_t c0, int32_t nchunks, int L, int32_t n,
                                 const int4 *__restrict__ meta, const int32_t *__restrict__ ecol,
                                 const double *__restrict__ eval,
                                 const int32_t *__restrict__ row_id,
                                 const double *__restrict__ diag,
                                 const int32_t *__restrict__ chunk_level, int32_t lev0,
                                 const int32_t *__restrict__ tlp, const int32_t *__restrict__ pos_of,
                                 int32_t P0, int32_t W, int32_t T, int32_t K, int32_t nr,
                                 const int64_t *__restrict__ aptr, int32_t *__restrict__ trow,
                                 double2 *__restrict__ tdiag, int32_t *__restrict__ tnn,
                                 int4 *__restrict__ term, int32_t *__restrict__ acol,
                                 double *__restrict__ aval) {
    const int32_t c = c0 + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (c >= nchunks) return;
    const int4 mt = meta[c];
    const int64_t stride = (int64_t)mt.y * L;
    const int32_t lstart = tlp[chunk_level[c] - lev0];
    for (int32_t k = 0; k < mt.y; ++k) {
        const int32_t p = mt.x + k - P0;
        const double d = diag[2 * (int64_t)(mt.x + k)];
        trow[p] = row_id[mt.x + k];
        tdiag[p] = make_double2(d, diag[2 * (int64_t)(mt.x + k) + 1]);
        bool scaled = true;
        for (int32_t t = 0; t < mt.z; ++t)
            for (int sl = 0; sl < L; ++sl) {
                const int64_t e = mt.w + t * stride + (int64_t)k * L + sl;
                const int32_t col = ecol[e];
                if (col == PAD_COL || col < -n || eval[e] == 0.0) continue;
                const double q = eval[e] / d;
                scaled = scaled && isfinite(q) && fabs(q) >= 2.2250738585072014e-308;
            }
        int64_t ai = aptr[p];
        int32_t ni = 0, far = 0;
        for (int32_t t = 0; t < mt.z; ++t)
            for (int sl = 0; sl < L; ++sl) {
                const int64_t e = mt.w + t * stride + (int64_t)k * L + sl;
                const int32_t col = ecol[e];
                if (col == PAD_COL || col < -n) continue;
                const double v = scaled ? eval[e] / d : eval[e];
                const int32_t q = col >= 0 ? pos_of[col] - P0 : -1;
                if (q >= 0) {
                    const bool nearby = lstart - q <= W - T;
                    if (!nearby) far |= 1 << ni;
                    const long long vb = __double_as_longlong(v);
                    term[(int64_t)ni * nr + p] = make_int4(nearby ? (q & (W - 1)) : col, 0,
                                                           (int)(vb & 0xFFFFFFFFll),
                                                           (int)(vb >> 32));
                    ++ni;
                } else {
                    acol[ai] = col;
                    aval[ai] = v;
                    ++ai;
                }
            }
        tnn[p] = ni | (far << 8) | (scaled ? 0 : kTailUnscaled);
        for (int32_t j = ni; j < K; ++j) term[(int64_t)j * nr + p] = make_int4(0, 0, 0, 0);
    }
}

}  // namespace

cudaError_t launch_expand_queries(int32_t nq, const int32_t *q_level, const int32_t *q_tgt,
                                  const int64_t *q_off, const int32_t *level_ptr,
                                  const int32_t *perm, int32_t *item_row, int32_t *item_tgt,
                                  int32_t *item_q, int32_t *item_pos, cudaStream_t s) {
    if (nq == 0) return cudaSuccess;
    expand_queries_kernel<<<nq, 128, 0, s>>>(nq, q_level, q_tgt, q_off, level_ptr, perm,
                                             item_row, item_tgt, item_q, item_pos);
    return cudaGetLastError();
}

cudaError_t launch_rewrite_count(int64_t nitems, const int32_t *item_row,
                                 const int32_t *item_tgt, const int32_t *item_q,
                                 const int32_t *row_ptr, const int32_t *col,
                                 const int32_t *level, int cap, int32_t *fill_out,
                                 unsigned long long *added, int32_t *overflow, int32_t *maxlen,
                                 int num_sms, cudaStream_t s) {
    if (nitems == 0) return cudaSuccess;
    size_t smem;
    const int w = warps_for_cap(cap, false, &smem);
    cudaError_t e = cudaFuncSetAttribute(rewrite_count_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t blocks = (nitems + w - 1) / w;
    const int64_t cap_blocks = (int64_t)num_sms * 32;
    if (blocks > cap_blocks) blocks = cap_blocks;
    rewrite_count_kernel<<<(unsigned)blocks, w * 32, smem, s>>>(
        nitems, item_row, item_tgt, item_q, row_ptr, col, level, cap, fill_out, added,
        overflow, maxlen);
    return cudaGetLastError();
}

cudaError_t launch_rewrite_numeric(int64_t nitems, const int32_t *item_row,
                                   const int32_t *item_tgt, const int64_t *out_off,
                                   const int32_t *row_ptr, const int32_t *col,
                                   const double *val, const int32_t *level, int cap,
                                   int32_t *out_col, double *out_val, int32_t *nb_out,
                                   DevStatus *st, int num_sms, cudaStream_t s) {
    if (nitems == 0) return cudaSuccess;
    size_t smem;
    const int w = warps_for_cap(cap, true, &smem);
    cudaError_t e = cudaFuncSetAttribute(rewrite_numeric_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t blocks = (nitems + w - 1) / w;
    const int64_t cap_blocks = (int64_t)num_sms * 32;
    if (blocks > cap_blocks) blocks = cap_blocks;
    rewrite_numeric_kernel<<<(unsigned)blocks, w * 32, smem, s>>>(
        nitems, item_row, item_tgt, out_off, row_ptr, col, val, level, cap, out_col, out_val,
        nb_out, st);
    return cudaGetLastError();
}

namespace {
// most off-diagonal terms of a row, per level
__global__ void level_max_kernel(int32_t n, const int32_t *__restrict__ level,
                                 const int32_t *__restrict__ offdeg, int32_t *out) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicMax(&out[level[i]], offdeg[i]);
}

// Weighted critical path, one new level of the solve structure per launch
// (every dependency lies in an earlier level, so its finish time is known):
// warp per chunk, each lane its entries of one row; x terms (col >= 0) are
// dependencies, b terms (col in [-n, -1]) and x terms count as the row's
// terms, unknowns of a CTA-local run (col < -n) are decoded to their row.
__global__ void critpath_level_kernel(int32_t c0, int32_t c1, int L, int32_t n,
                                      const int4 *__restrict__ meta,
                                      const int32_t *__restrict__ ecol,
                                      const int32_t *__restrict__ row_id,
                                      const int32_t *__restrict__ chunk_run_p0, int64_t hop,
                                      int64_t *finish) {
    const int64_t c = c0 + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= c1) return;
    const int4 mt = meta[c];
    const int k = lane / L, s = lane % L;
    int64_t terms = 0, dep = 0;
    if (k < mt.y) {
        const int64_t stride = (int64_t)mt.y * L;
        for (int j = s; j < mt.z * L; j += L) {
            int32_t cc = ecol[mt.w + (int64_t)(j / L) * stride + (int64_t)k * L + (j % L)];
            if (cc == PAD_COL) continue;
            ++terms;
            if (cc < -n && chunk_run_p0) cc = row_id[chunk_run_p0[c] + (-(n + 1) - cc)];
            if (cc >= 0) dep = max(dep, finish[cc]);
        }
    }
    for (int o = L / 2; o > 0; o >>= 1) {
        terms += __shfl_xor_sync(FULL_MASK, terms, o);
        dep = max(dep, __shfl_xor_sync(FULL_MASK, dep, o));
    }
    if (k < mt.y && s == 0) finish[row_id[mt.x + k]] = hop + terms + dep;
}
}  // namespace

namespace {
// Per-level counts of the analysis features: acc[l][0] rows, [1] entries,
// [2 + b] rows in log2 length bin b, [10] ancestor span (max).
__global__ void level_counts_kernel(int32_t n, const int32_t *__restrict__ row_ptr,
                                    const int32_t *__restrict__ col,
                                    const int32_t *__restrict__ level,
                                    unsigned long long *acc) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t a = row_ptr[i], e = row_ptr[i + 1] - 1;   // the diagonal is last
    const int32_t c = e - a;
    const int32_t lv = level[i];
    int32_t lo = lv;
    for (int32_t k = a; k < e; ++k) lo = min(lo, level[col[k]]);
    const int bin = c <= 0 ? 0 : min(32 - __clz(c), 7);
    unsigned long long *q = acc + (int64_t)lv * 11;
    atomicAdd(&q[0], 1ull);
    atomicAdd(&q[1], (unsigned long long)c);
    atomicAdd(&q[2 + bin], 1ull);
    atomicMax(&q[10], (unsigned long long)(lv - lo));
}
}  // namespace

cudaError_t launch_level_counts(int32_t n, const int32_t *row_ptr, const int32_t *col,
                                const int32_t *level, unsigned long long *acc, cudaStream_t s) {
    if (n > 0)
        level_counts_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, row_ptr, col, level, acc);
    return cudaGetLastError();
}

cudaError_t launch_level_max(int32_t n, const int32_t *level, const int32_t *offdeg, int32_t *out,
                             cudaStream_t s) {
    if (n > 0) level_max_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, level, offdeg, out);
    return cudaGetLastError();
}

cudaError_t launch_critpath_level(int32_t c0, int32_t c1, int L, int32_t n, const int4 *meta,
                                  const int32_t *ecol, const int32_t *row_id,
                                  const int32_t *chunk_run_p0, int64_t hop, int64_t *finish,
                                  cudaStream_t s) {
    if (c1 <= c0) return cudaSuccess;
    const int64_t threads = (int64_t)(c1 - c0) * 32;
    critpath_level_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        c0, c1, L, n, meta, ecol, row_id, chunk_run_p0, hop, finish);
    return cudaGetLastError();
}

cudaError_t launch_pos_item(int32_t n, int64_t nitems, const int32_t *item_pos,
                            int32_t *pos_item, cudaStream_t s) {
    if (n > 0) fill_i32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pos_item, n, -1);
    if (nitems > 0)
        scatter_item_index<<<(unsigned)((nitems + 255) / 256), 256, 0, s>>>(nitems, item_pos,
                                                                           pos_item);
    return cudaGetLastError();
}

cudaError_t launch_chunk_width(int32_t nchunks, const int32_t *c_row0, const int32_t *c_nrows,
                               int L, const int32_t *perm, const int32_t *offdeg,
                               const int32_t *pos_item, const int64_t *rw_off, int64_t *slots,
                               int32_t *width, cudaStream_t s) {
    if (nchunks == 0) return cudaSuccess;
    chunk_width_kernel<<<(nchunks + 255) / 256, 256, 0, s>>>(nchunks, c_row0, c_nrows, L, perm,
                                                             offdeg, pos_item, rw_off, slots,
                                                             width);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_chunk_fill(int32_t nchunks, int L, const int32_t *c_row0,
                              const int32_t *c_nrows, const int32_t *c_width,
                              const int64_t *c_off, const int32_t *perm, const int32_t *row_ptr,
                              const int32_t *col, const double *val, const int32_t *pos_item,
                              const int64_t *rw_off, const int32_t *rw_col,
                              const double *rw_val, int4 *meta, int32_t *ecol, T *eval,
                              int32_t *row_id, T *diag, cudaStream_t s) {
    if (nchunks == 0) return cudaSuccess;
    const int H = 32 / L;
    const int64_t threads = (int64_t)nchunks * H;
    chunk_fill_kernel<T><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        nchunks, H, L, c_row0, c_nrows, c_width, c_off, perm, row_ptr, col, val, pos_item,
        rw_off, rw_col, rw_val, meta, ecol, eval, row_id, diag);
    return cudaGetLastError();
}
template cudaError_t launch_chunk_fill<double>(int32_t, int, const int32_t *, const int32_t *,
                                               const int32_t *, const int64_t *,
                                               const int32_t *, const int32_t *,
                                               const int32_t *, const double *,
                                               const int32_t *, const int64_t *,
                                               const int32_t *, const double *, int4 *,
                                               int32_t *, double *, int32_t *, double *,
                                               cudaStream_t);
template cudaError_t launch_chunk_fill<float>(int32_t, int, const int32_t *, const int32_t *,
                                              const int32_t *, const int64_t *,
                                              const int32_t *, const int32_t *,
                                              const int32_t *, const double *,
                                              const int32_t *, const int64_t *,
                                              const int32_t *, const double *, int4 *,
                                              int32_t *, float *, int32_t *, float *,
                                              cudaStream_t);

cudaError_t launch_export_count(int32_t nchunks, int L, const int4 *meta, const int32_t *ecol,
                                const int32_t *row_id, int32_t n, int64_t *xcnt, int64_t *bcnt,
                                cudaStream_t s) {
    if (nchunks == 0) return cudaSuccess;
    const int H = 32 / L;
    const int64_t threads = (int64_t)nchunks * H;
    export_count_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        nchunks, H, L, meta, ecol, row_id, n, xcnt, bcnt);
    return cudaGetLastError();
}

cudaError_t launch_export_fill(int32_t nchunks, int L, const int4 *meta, const int32_t *ecol,
                               const double *eval, const int32_t *row_id,
                               const int32_t *chunk_level, const int32_t *chunk_run_p0,
                               int32_t n, const int64_t *xptr, const int64_t *bptr,
                               int32_t *xcol, double *xval, int32_t *bcol, double *bw,
                               int32_t *new_level, cudaStream_t s) {
    if (nchunks == 0) return cudaSuccess;
    const int H = 32 / L;
    const int64_t threads = (int64_t)nchunks * H;
    export_fill_kernel<double><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        nchunks, H, L, meta, ecol, eval, row_id, chunk_level, chunk_run_p0, n, xptr, bptr, xcol,
        xval, bcol, bw, new_level);
    return cudaGetLastError();
}

cudaError_t launch_chunk_level(int32_t nlev, const int32_t *lvl_chunk, int32_t *chunk_level,
                               cudaStream_t s) {
    if (nlev == 0) return cudaSuccess;
    chunk_level_kernel<<<nlev, 128, 0, s>>>(nlev, lvl_chunk, chunk_level);
    return cudaGetLastError();
}

cudaError_t launch_encode_runs(int32_t n, int L, const int32_t *row_id, const int4 *meta,
                               int32_t nrc, const int32_t *run_chunk, const int2 *run_span,
                               int32_t *pos_tmp, int32_t *ecol, cudaStream_t s) {
    if (n == 0 || nrc == 0) return cudaSuccess;
    pos_of_row_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, row_id, pos_tmp);
    const int H = 32 / L;
    const int64_t threads = (int64_t)nrc * H;
    encode_run_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(nrc, run_chunk, run_span, H,
                                                                       L, n, meta, pos_tmp, ecol);
    return cudaGetLastError();
}

cudaError_t launch_f64_to_f32(const double *a, float *b, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    f64_to_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, b, n);
    return cudaGetLastError();
}

cudaError_t launch_pos_of_row(int32_t n, const int32_t *row_id, int32_t *pos, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    pos_of_row_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, row_id, pos);
    return cudaGetLastError();
}

cudaError_t launch_tail_count(int32_t c0, int32_t nchunks, int L, int32_t n, const int4 *meta,
                              const int32_t *ecol, const int32_t *pos_of, int32_t P0,
                              int32_t *cnt_a, int32_t *cnt_n, int32_t *kmax, int32_t *bad,
                              cudaStream_t s) {
    const int32_t m = nchunks - c0;
    if (m <= 0) return cudaSuccess;
    tail_count_kernel<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(c0, nchunks, L, n, meta, ecol,
                                                                  pos_of, P0, cnt_a, cnt_n,
                                                                  kmax, bad);
    return cudaGetLastError();
}

cudaError_t launch_tail_fill(int32_t c0, int32_t nchunks, int L, int32_t n, const int4 *meta,
                             const int32_t *ecol, const double *eval, const int32_t *row_id,
                             const double *diag, const int32_t *chunk_level, int32_t lev0,
                             const int32_t *tlp, const int32_t *pos_of, int32_t P0, int32_t W,
                             int32_t T, int32_t K, int32_t nr, const int64_t *aptr,
                             int32_t *trow, double2 *tdiag, int32_t *tnn, int4 *term,
                             int32_t *acol, double *aval, cudaStream_t s) {
    const int32_t m = nchunks - c0;
    if (m <= 0) return cudaSuccess;
    tail_fill_kernel<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(
        c0, nchunks, L, n, meta, ecol, eval, row_id, diag, chunk_level, lev0, tlp, pos_of, P0, W,
        T, K, nr, aptr, trow, tdiag, tnn, term, acol, aval);
    return cudaGetLastError();
}

}  // namespace sptrsv
