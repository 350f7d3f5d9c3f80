// Solve kernels over the level-ordered structure built by the transform.
//
// Level-set execution (Sec. II): rows of a level run in parallel, levels run
// in sequence.  Two kernels share one chunk processor:
//  * solve_barrier_kernel: a persistent, co-resident grid walks the schedule
//    of phases; a phase is either one level processed by the whole grid, or a
//    run of consecutive thin levels processed by a single CTA with
//    __syncthreads between levels (no grid-wide synchronisation inside the
//    run).  A grid barrier separates phases.
//  * solve_syncfree_kernel: the synchronisation-free alternative of Sec. II
//    (rows wait for their own dependencies only).  Chunks are taken in level
//    order by a persistent grid; every unknown is pre-set to a signalling-NaN
//    sentinel and a lane spins (bounded) on the unknowns it reads until they
//    hold computed values, so the value is its own ready flag and no fence
//    is needed between producer and consumer.
// Every lane of a chunk handles one row (L lanes per row for long rows,
// summed by shuffles) or, with several right-hand sides, one (row, column).
#include "solve.cuh"

namespace sptrsv {
namespace {

template <typename T> struct Bits;
template <> struct Bits<double> {
    using U = unsigned long long;
    static __device__ __forceinline__ U load(const double *p) { return ld_relaxed_u64(p); }
    static __device__ __forceinline__ U poll(const double *p) {
        U v;
        asm volatile("ld.volatile.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
        return v;
    }
    static __device__ __forceinline__ void store(double *p, double v) {
        U b = (U)__double_as_longlong(v);
        if (b == Sentinel<double>::bits) b = 0x7FF8000000000000ull;
        st_relaxed_u64(p, b);
    }
    static __device__ __forceinline__ double from(U b) { return __longlong_as_double((long long)b); }
    static __device__ __forceinline__ U of(double v) { return (U)__double_as_longlong(v); }
};
template <> struct Bits<float> {
    using U = unsigned;
    static __device__ __forceinline__ U load(const float *p) { return ld_relaxed_u32(p); }
    static __device__ __forceinline__ U poll(const float *p) {
        U v;
        asm volatile("ld.volatile.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
        return v;
    }
    static __device__ __forceinline__ void store(float *p, float v) {
        U b = __float_as_uint(v);
        if (b == Sentinel<float>::bits) b = 0x7FC00000u;
        st_relaxed_u32(p, b);
    }
    static __device__ __forceinline__ float from(U b) { return __uint_as_float(b); }
    static __device__ __forceinline__ U of(float v) { return __float_as_uint(v); }
};

// Value of an unknown written by another warp of this launch.
template <typename T, bool SF>
__device__ __forceinline__ T load_x(const T *p) {
    if (SF) return Bits<T>::from(Bits<T>::poll(p));
    return __ldcg(p);
}

// Bounded spin until *p holds a computed value (synchronisation-free only).
// Returns the value's bits; the sentinel's bits mean the wait gave up (a
// computed value never has them: stores turn them into a quiet NaN).  The
// out-of-line copy keeps the spin loop out of the hot path, and returning
// the status by value keeps the caller's flag in a register.
template <typename T>
__device__ __forceinline__ typename Bits<T>::U wait_bits_inl(const T *p, DevStatus *st,
                                                            uint64_t timeout_ns, int backoff_ns) {
    WaitBudget wb(timeout_ns);
    unsigned it = 0;
    typename Bits<T>::U b;
    do {
        if (backoff_ns) __nanosleep(backoff_ns);
        if ((++it & kPollMask) == 0 && wb.expired(st, -2)) return Sentinel<T>::bits;
        b = Bits<T>::poll(p);
    } while (b == Sentinel<T>::bits);
    return b;
}
template <typename T>
__device__ __noinline__ typename Bits<T>::U wait_bits(const T *p, DevStatus *st,
                                                     uint64_t timeout_ns, int backoff_ns) {
    return wait_bits_inl<T>(p, st, timeout_ns, backoff_ns);
}
template <typename T>
__device__ __forceinline__ T bits_or_bail(typename Bits<T>::U b, bool &bail) {
    if (b == Sentinel<T>::bits) {
        bail = true;
        return T(0);
    }
    return Bits<T>::from(b);
}
template <typename T>
__device__ __forceinline__ T wait_x(const T *p, DevStatus *st, uint64_t timeout_ns,
                                    int backoff_ns, bool &bail) {
    return bits_or_bail<T>(wait_bits<T>(p, st, timeout_ns, backoff_ns), bail);
}
template <typename T>
__device__ __forceinline__ T wait_x_inl(const T *p, DevStatus *st, uint64_t timeout_ns,
                                        int backoff_ns, bool &bail) {
    return bits_or_bail<T>(wait_bits_inl<T>(p, st, timeout_ns, backoff_ns), bail);
}

template <typename T, bool SF>
__device__ __forceinline__ void store_x(T *p, T v) {
    if (SF) Bits<T>::store(p, v);
    else *p = v;
}

// Division by the diagonal without an FP64/FP32 divide on the common path.
// With y = RN(1/d) precomputed (0 when d lies outside the safe range),
// q = RN(s y) is within an ulp of s/d, the remainder r = s - d q is exact
// (one FMA), and RN(q + r y) is the correctly rounded quotient (Markstein,
// "Computation of elementary functions on the IBM RISC System/6000
// processor", IBM J. Res. Dev. 1990).  The argument needs the remainder to be
// representable, so the numerator must stay well above the subnormal range
// (|s| in [slo, shi)) and the result away from underflow and overflow
// (|q| in [qlo, qhi)); everything else takes an IEEE division.
template <typename T> struct DivRange;
template <> struct DivRange<double> {  // bit patterns of 2^-900, 2^900, 2^-1000, 2^1000
    static constexpr unsigned long long abs = 0x7FFFFFFFFFFFFFFFull;
    static constexpr unsigned long long slo = 0x07B0000000000000ull, shi = 0x7830000000000000ull;
    static constexpr unsigned long long qlo = 0x0170000000000000ull, qhi = 0x7E70000000000000ull;
};
template <> struct DivRange<float> {  // bit patterns of 2^-100, 2^100, 2^-120, 2^120
    static constexpr unsigned abs = 0x7FFFFFFFu;
    static constexpr unsigned slo = 0x0D800000u, shi = 0x71800000u;
    static constexpr unsigned qlo = 0x03800000u, qhi = 0x7B800000u;
};

// The range tests compare bit patterns as integers (for non-negative
// floating-point numbers the order is the same, and NaN lies above every
// bound), which keeps them off the FP64 pipe: on this GPU every FP64
// instruction is a scarce resource.
template <typename T>
__device__ __forceinline__ T div_by_diag(T s, T d, T y) {
    using R = DivRange<T>;
    const auto as = Bits<T>::of(s) & R::abs;
    if (Bits<T>::of(y) != 0 && as - R::slo < R::shi - R::slo) {
        const T q = s * y;
        const T r = fma(-q, d, s);
        const T q2 = fma(r, y, q);
        const auto a = Bits<T>::of(q2) & R::abs;
        if (a - R::qlo < R::qhi - R::qlo) return q2;
    }
    return s / d;
}

template <typename T> struct Vec2;
template <> struct Vec2<double> { using V = double2; };
template <> struct Vec2<float> { using V = float2; };

template <typename T>
__device__ __forceinline__ void load_diag(const SolveData<T> &sd, int32_t p, T &d, T &y) {
    const typename Vec2<T>::V v = __ldg(reinterpret_cast<const typename Vec2<T>::V *>(sd.diag) + p);
    d = v.x;
    y = v.y;
}

struct Ctx {
    const double *rhs;
    int ld;
    int nr;
    DevStatus *st;
    uint64_t timeout_ns;
    int backoff_ns;
    bool rhs_coherent;   // rhs was written earlier in this launch: read it through L2
    int32_t n;           // rows (decodes b terms and run slots)
    const int32_t *row_id;
    void *xs;            // shared-memory unknowns of the current CTA-local run, or null
    int32_t run_p0;      // first solve position of the current run
};

__device__ __forceinline__ double load_rhs(const Ctx &cx, int64_t i) {
    return cx.rhs_coherent ? __ldcg(cx.rhs + i) : __ldg(cx.rhs + i);
}

// A term that is not an unknown of another CTA: a b term of a rewritten row
// (col = ~j), a padding slot, or -- inside a CTA-local run -- an unknown of
// the same run (col = -(n + 1) - slot, kept in shared memory; the
// several-right-hand-side path reads it back from x through L2).
template <typename T>
__device__ __forceinline__ T other_term(const Ctx &cx, int32_t c, const T *out, int r) {
    if (c >= -cx.n) return (T)load_rhs(cx, (int64_t)(~c) * cx.ld + r);
    if (c == PAD_COL) return T(0);
    const int32_t slot = -(cx.n + 1) - c;
    if (cx.xs) return reinterpret_cast<const T *>(cx.xs)[slot];
    return __ldcg(out + (int64_t)__ldg(&cx.row_id[cx.run_p0 + slot]) * cx.ld + r);
}

template <typename T>
__device__ __forceinline__ void keep_in_run(const Ctx &cx, int32_t pos, T v) {
    if (cx.xs) reinterpret_cast<T *>(cx.xs)[pos - cx.run_p0] = v;
}

// One right-hand side; L lanes per row (compile time).
// U consecutive steps of one lane's entries: U entry loads, then U x (or b)
// loads in flight together, then the terms already computed and, last, the
// late arrivals, each one dependent FMA on a sum that starts at b_i.
template <typename T, int U, bool SF>
__device__ __forceinline__ void row_batch(const int32_t *cp, const T *vp, int64_t stride, int step,
                                          T *out, const Ctx &cx, T &acc, bool &bail) {
    int32_t cc[U];
    T vv[U], xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        cc[u] = __ldg(cp + (int64_t)(step + u) * stride);
        vv[u] = __ldg(vp + (int64_t)(step + u) * stride);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (cc[u] >= 0) xv[u] = load_x<T, SF>(out + (int64_t)cc[u] * cx.ld);
        else xv[u] = other_term<T>(cx, cc[u], out, 0);
    }
    bool pend[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        pend[u] = SF && cc[u] >= 0 && Bits<T>::of(xv[u]) == Sentinel<T>::bits;
        if (!pend[u]) acc = fma(-vv[u], xv[u], acc);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
        if (pend[u])
            acc = fma(-vv[u],
                      wait_x<T>(out + (int64_t)cc[u] * cx.ld, cx.st, cx.timeout_ns, cx.backoff_ns,
                                bail),
                      acc);
}

template <typename T, int L, bool SF>
__device__ __forceinline__ bool chunk_one(const SolveData<T> &sd, int32_t c, T *out,
                                          const Ctx &cx) {
    const int lane = threadIdx.x & 31;
    const int k = lane / L, s = lane % L;
    const int4 mt = __ldg(&sd.meta[c]);
    const bool active = k < mt.y;
    T acc = T(0);
    bool bail = false;
    int32_t r = 0;
    T brow = T(0), dg = T(1), dy = T(1);
    if (active && s == 0) {  // independent of every unknown: issue first
        r = __ldg(&sd.row_id[mt.x + k]);
        load_diag<T>(sd, mt.x + k, dg, dy);
        brow = (T)load_rhs(cx, (int64_t)r * cx.ld);
        acc = brow;
    }
    if (active) {
        const int64_t stride = (int64_t)mt.y * L;
        const int32_t *cp = sd.ecol + mt.w + k * L + s;
        const T *vp = sd.eval + mt.w + k * L + s;
        int step = 0;
        for (; step + 4 <= mt.z; step += 4)
            row_batch<T, 4, SF>(cp, vp, stride, step, out, cx, acc, bail);
        switch (mt.z - step) {  // the remainder as one batch of its exact size
        case 3: row_batch<T, 3, SF>(cp, vp, stride, step, out, cx, acc, bail); step += 3; break;
        case 2: row_batch<T, 2, SF>(cp, vp, stride, step, out, cx, acc, bail); step += 2; break;
        case 1: row_batch<T, 1, SF>(cp, vp, stride, step, out, cx, acc, bail); step += 1; break;
        default: break;
        }
        for (; step < mt.z; ++step) {
            const int32_t cc = __ldg(cp + (int64_t)step * stride);
            const T v = __ldg(vp + (int64_t)step * stride);
            T xv = T(0);
            if (cc >= 0) {
                xv = load_x<T, SF>(out + (int64_t)cc * cx.ld);
                if (SF && Bits<T>::of(xv) == Sentinel<T>::bits)
                    xv = wait_x<T>(out + (int64_t)cc * cx.ld, cx.st, cx.timeout_ns, cx.backoff_ns, bail);
            } else {
                xv = other_term<T>(cx, cc, out, 0);
            }
            acc = fma(-v, xv, acc);
        }
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL_MASK, acc, o);
    if (active && s == 0) {
        const T res = div_by_diag<T>(acc, dg, dy);
        store_x<T, SF>(out + (int64_t)r * cx.ld, res);
        keep_in_run<T>(cx, mt.x + k, res);
    }
    return __any_sync(FULL_MASK, bail);
}

// Several right-hand sides: R lanes per row, lane r owns column r.
template <typename T, int R, bool SF>
__device__ __forceinline__ bool chunk_multi(const SolveData<T> &sd, int32_t c, T *out,
                                            const Ctx &cx) {
    constexpr int G = 32 / R;
    const int lane = threadIdx.x & 31;
    const int g = lane / R, r = lane % R;
    const int4 mt = __ldg(&sd.meta[c]);
    const int L = sd.L;
    const int64_t stride = (int64_t)mt.y * L;
    bool bail = false;
    for (int kb = 0; kb < mt.y; kb += G) {
        const int k = kb + g;
        const bool rowok = k < mt.y;
        const bool active = rowok && r < cx.nr;
        T acc = T(0);
        int32_t row = 0;
        T brow = T(0), dg = T(1), dy = T(1);
        if (active) {  // independent of every unknown: issue first
            row = __ldg(&sd.row_id[mt.x + k]);
            load_diag<T>(sd, mt.x + k, dg, dy);
            brow = (T)load_rhs(cx, (int64_t)row * cx.ld + r);
            acc = brow;
        }
        if (active) {
            // the row's entries in storage order, U at a time: U loads of
            // entries, then U loads of x (or b) values in flight together,
            // then the waits and FMAs (terms already computed first)
            const int64_t base = mt.w + (int64_t)k * L;
            const int nent = mt.z * L;
            auto slot_of = [&](int j) { return base + (int64_t)(j / L) * stride + (j % L); };
            constexpr int U = 4;
            int j = 0;
            for (; j + U <= nent; j += U) {
                int32_t cc[U];
                T vv[U], xv[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t sl = slot_of(j + u);
                    cc[u] = __ldg(sd.ecol + sl);
                    vv[u] = __ldg(sd.eval + sl);
                }
                if (cc[0] == PAD_COL) break;  // a row's entries come first, pads after
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (cc[u] >= 0) xv[u] = load_x<T, SF>(out + (int64_t)cc[u] * cx.ld + r);
                    else xv[u] = other_term<T>(cx, cc[u], out, r);
                }
                bool pend[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    pend[u] = SF && cc[u] >= 0 && Bits<T>::of(xv[u]) == Sentinel<T>::bits;
                    if (!pend[u]) acc = fma(-vv[u], xv[u], acc);
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (pend[u])
                        acc = fma(-vv[u],
                                  wait_x<T>(out + (int64_t)cc[u] * cx.ld + r, cx.st,
                                            cx.timeout_ns, cx.backoff_ns, bail),
                                  acc);
            }
            for (; j < nent; ++j) {
                const int64_t sl = slot_of(j);
                const int32_t cc = __ldg(sd.ecol + sl);
                if (cc == PAD_COL) break;
                const T v = __ldg(sd.eval + sl);
                T xv;
                if (cc >= 0) {
                    T *px = out + (int64_t)cc * cx.ld + r;
                    xv = load_x<T, SF>(px);
                    if (SF && Bits<T>::of(xv) == Sentinel<T>::bits)
                        xv = wait_x<T>(px, cx.st, cx.timeout_ns, cx.backoff_ns, bail);
                } else {
                    xv = other_term<T>(cx, cc, out, r);
                }
                acc = fma(-v, xv, acc);
            }
        }
        if (active)
            store_x<T, SF>(out + (int64_t)row * cx.ld + r, div_by_diag<T>(acc, dg, dy));
        if (__any_sync(FULL_MASK, bail)) return true;
    }
    return false;
}


// ---------------------------------------------------------------------------
// Software pipeline for one right-hand side: a chunk's entries are loaded
// into registers (stage_entries) one chunk ahead, so that when the chunk is
// finished only the gather of its b and x values (one round trip) and the
// wait for its dependencies remain.  Chunks wider than kPipeSteps entries
// per lane go through chunk_one.
constexpr int kPipeSteps = 4;
// Largest CTA of the solve kernels: 512 threads leave 128 registers per
// thread, enough for the staged chunk without spilling.
constexpr int kMaxSolveThreads = 512;

template <typename T>
struct Staged {
    int4 mt;
    int32_t col[kPipeSteps];
    T val[kPipeSteps];
    int32_t row;   // row of this lane's chunk row (lane s == 0 only)
    T diag, rdiag;
};

template <typename T, int L>
__device__ __forceinline__ void stage_entries(const SolveData<T> &sd, Staged<T> &sg) {
    const int lane = threadIdx.x & 31;
    const int k = lane / L, s = lane % L;
    const bool ok = k < sg.mt.y && sg.mt.z <= kPipeSteps;
    const int64_t stride = (int64_t)sg.mt.y * L;
    const int64_t base = (int64_t)sg.mt.w + k * L + s;
#pragma unroll
    for (int u = 0; u < kPipeSteps; ++u) {
        if (ok && u < sg.mt.z) {
            sg.col[u] = __ldg(sd.ecol + base + u * stride);
            sg.val[u] = __ldg(sd.eval + base + u * stride);
        } else {
            sg.col[u] = PAD_COL;
            sg.val[u] = T(0);
        }
    }
    // the row and its diagonal do not depend on any unknown: load them now
    if (k < sg.mt.y && s == 0) {
        sg.row = __ldg(&sd.row_id[sg.mt.x + k]);
        load_diag<T>(sd, sg.mt.x + k, sg.diag, sg.rdiag);
    } else {
        sg.row = 0;
        sg.diag = T(1);
        sg.rdiag = T(1);
    }
}

template <typename T, int L, bool SF>
__device__ __forceinline__ bool finish_staged(const SolveData<T> &sd, const Staged<T> &sg,
                                              T *out, const Ctx &cx) {
    const int lane = threadIdx.x & 31;
    const int k = lane / L, s = lane % L;
    const bool active = k < sg.mt.y;
    // b_i first: nothing after the wait may be another dependent load
    const T brow = (active && s == 0) ? (T)load_rhs(cx, (int64_t)sg.row * cx.ld) : T(0);
    T xv[kPipeSteps];
#pragma unroll
    for (int u = 0; u < kPipeSteps; ++u) {
        const int32_t c = sg.col[u];
        if (c >= 0) xv[u] = load_x<T, SF>(out + (int64_t)c * cx.ld);
        else xv[u] = other_term<T>(cx, c, out, 0);
    }
    bool bail = false;
    // the sum runs from b_i down, one FMA per staged step (FP64 instructions
    // are the scarce resource: no separate products, no tree)
    T acc = brow;
#pragma unroll
    for (int u = 0; u < kPipeSteps; ++u) {
        if (u >= sg.mt.z) break;
        if (SF && sg.col[u] >= 0 && Bits<T>::of(xv[u]) == Sentinel<T>::bits)
            xv[u] = wait_x_inl<T>(out + (int64_t)sg.col[u] * cx.ld, cx.st, cx.timeout_ns,
                                  cx.backoff_ns, bail);
        acc = fma(-sg.val[u], xv[u], acc);
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL_MASK, acc, o);
    if (active && s == 0) {
        const T res = div_by_diag<T>(acc, sg.diag, sg.rdiag);
        store_x<T, SF>(out + (int64_t)sg.row * cx.ld, res);
        keep_in_run<T>(cx, sg.mt.x + k, res);
    }
    return __any_sync(FULL_MASK, bail);
}

template <typename T, int L, bool SF>
__device__ __forceinline__ bool finish_any(const SolveData<T> &sd, int32_t c,
                                           const Staged<T> &sg, T *out, const Ctx &cx) {
    if (sg.mt.z > kPipeSteps) return chunk_one<T, L, SF>(sd, c, out, cx);
    return finish_staged<T, L, SF>(sd, sg, out, cx);
}

template <typename T, int L>
__device__ __forceinline__ void stage_chunk(const SolveData<T> &sd, int32_t c, Staged<T> &sg) {
    sg.mt = __ldg(&sd.meta[c]);
    stage_entries<T, L>(sd, sg);
}

template <typename T, int L, int R, bool SF>
__device__ __forceinline__ bool process_chunk(const SolveData<T> &sd, int32_t c, T *out,
                                              const Ctx &cx) {
    if (R == 1) return chunk_one<T, L, SF>(sd, c, out, cx);
    return chunk_multi<T, R, SF>(sd, c, out, cx);
}

__device__ __forceinline__ bool converged(const DevStatus *st) {
    return ld_relaxed_u64(&st->ir_flag) != 0ull;
}

// Start of every solve kernel: pull the arrays that are read by row (meta,
// row_id, diag) and the right-hand side into L2, so that gathers from them
// hit L2 instead of HBM.  The rhs prefetch is capped at 64 MiB.
template <typename T>
__device__ __forceinline__ void prefetch_solve_inputs(const SolveData<T> &sd, const double *rhs,
                                                      int64_t n, int ld, int nr) {
    l2_prefetch_slice(sd.meta, (size_t)sd.nchunks * sizeof(int4));
    l2_prefetch_slice(sd.row_id, (size_t)n * sizeof(int32_t));
    l2_prefetch_slice(sd.diag, (size_t)n * 2 * sizeof(T));
    // rhs points at column c0 of a row-major [n, ld] array: the last element
    // this launch reads is ((n - 1) * ld + nr - 1), so stay inside that
    if (n <= 0) return;
    size_t rb = ((size_t)(n - 1) * ld + nr) * sizeof(double);
    if (rb > (64u << 20)) rb = 64u << 20;
    l2_prefetch_slice(rhs, rb);
}

// The warp's first chunk of phase ph (or -1): fat levels are shared by the
// whole grid, a CTA-local run belongs to CTA ph % gridDim.x.
template <typename T>
__device__ __forceinline__ int32_t first_chunk_of_phase(const SolveData<T> &sd, int ph,
                                                        int32_t gw, int wib) {
    if (ph >= sd.nphases) return -1;
    const int2 p = __ldg(&sd.phases[ph]);
    if (p.y > 0) {
        const int32_t c = __ldg(&sd.lvl_chunk[p.x]) + gw;
        return c < __ldg(&sd.lvl_chunk[p.x + 1]) ? c : -1;
    }
    if ((int)blockIdx.x != ph % (int)gridDim.x) return -1;
    const int32_t c = __ldg(&sd.lvl_chunk[p.x]) + wib;
    return c < __ldg(&sd.lvl_chunk[p.x + 1]) ? c : -1;
}

// The chunks one warp of a synchronisation-free launch solves, in order:
// the level-major schedule when it was dealt to this many warps, else every
// nw-th chunk.  Chunks at or past sd.nchunks (a tail solved by another
// kernel) end the sequence: they come after all others in both orders.
struct WarpChunks {
    const int32_t *list;   // schedule slice of this warp, or null
    int32_t count;
    int32_t gw, nw, nchunks;
    __device__ __forceinline__ int32_t at(int32_t j) const {
        if (list) {
            if (j >= count) return -1;
            const int32_t c = __ldg(list + j);
            return c < nchunks ? c : -1;
        }
        const int64_t c = (int64_t)gw + (int64_t)j * nw;
        return c < nchunks ? (int32_t)c : -1;
    }
};
template <typename T>
__device__ __forceinline__ WarpChunks warp_chunks(const SolveData<T> &sd, int32_t gw, int32_t nw) {
    if (sd.sched && sd.sched_nw == nw) {
        const int32_t a = __ldg(sd.sched_ptr + gw), b = __ldg(sd.sched_ptr + gw + 1);
        return WarpChunks{sd.sched + a, b - a, gw, nw, sd.nchunks};
    }
    return WarpChunks{nullptr, 0, gw, nw, sd.nchunks};
}

template <typename T, int L, int R>
__global__ void __launch_bounds__(kMaxSolveThreads)
solve_barrier_kernel(SolveData<T> sd, const double *rhs, T *out, int ld, int nr,
                     DevStatus *st, uint64_t timeout_ns, int skip_if_converged) {
    if (skip_if_converged && converged(st)) return;  // uniform: set by an earlier kernel
    extern __shared__ __align__(16) unsigned char run_smem[];
    const Ctx cx{rhs, ld, nr, st, timeout_ns, 0, false, sd.n, sd.row_id, nullptr, 0};
    const int wpb = blockDim.x >> 5, wib = threadIdx.x >> 5;
    const int32_t gw = blockIdx.x * wpb + wib;
    const int32_t nw = gridDim.x * wpb;
    unsigned long long bar = 0;
    prefetch_solve_inputs<T>(sd, rhs, sd.n, ld, nr);
    // One right-hand side: the warp's first chunk of the next phase (or of
    // the next level of a run) is staged before the barrier that precedes it.
    Staged<T> sg;
    int32_t staged = -1;
    if (R == 1) {
        staged = first_chunk_of_phase<T>(sd, 0, gw, wib);
        if (staged >= 0) stage_chunk<T, L>(sd, staged, sg);
    }
    for (int ph = 0; ph < sd.nphases; ++ph) {
        const int2 p = __ldg(&sd.phases[ph]);
        if (p.y > 0) {
            const int32_t c1 = __ldg(&sd.lvl_chunk[p.x + 1]);
            for (int32_t c = __ldg(&sd.lvl_chunk[p.x]) + gw; c < c1; c += nw) {
                if (R == 1 && c == staged) finish_any<T, L, false>(sd, c, sg, out, cx);
                else process_chunk<T, L, R, false>(sd, c, out, cx);
            }
        } else if ((int)blockIdx.x == ph % (int)gridDim.x) {
            // CTA-local run: its unknowns also go to shared memory, where the
            // run's later levels read them
            Ctx rc = cx;
            rc.run_p0 = __ldg(&sd.meta[__ldg(&sd.lvl_chunk[p.x])]).x;
            rc.xs = (R == 1 && sd.run_slots > 0) ? (void *)run_smem : nullptr;
            for (int32_t l = p.x; l < -p.y; ++l) {
                const int32_t c1 = __ldg(&sd.lvl_chunk[l + 1]);
                for (int32_t c = __ldg(&sd.lvl_chunk[l]) + wib; c < c1; c += wpb) {
                    if (R == 1 && c == staged) finish_any<T, L, false>(sd, c, sg, out, rc);
                    else process_chunk<T, L, R, false>(sd, c, out, rc);
                }
                if (R == 1 && l + 1 < -p.y) {
                    const int32_t c = __ldg(&sd.lvl_chunk[l + 1]) + wib;
                    staged = c < __ldg(&sd.lvl_chunk[l + 2]) ? c : -1;
                    if (staged >= 0) stage_chunk<T, L>(sd, staged, sg);
                }
                __syncthreads();
            }
        }
        if (ph + 1 < sd.nphases) grid_arrive(st);
        if (R == 1) {
            staged = first_chunk_of_phase<T>(sd, ph + 1, gw, wib);
            if (staged >= 0) stage_chunk<T, L>(sd, staged, sg);
        }
        if (ph + 1 < sd.nphases && !grid_wait(st, (++bar) * gridDim.x, timeout_ns, ph)) break;
    }
    grid_exit(st);
}

template <typename T, int L, int R>
__global__ void __launch_bounds__(kMaxSolveThreads)
solve_syncfree_kernel(SolveData<T> sd, const double *rhs, T *out, int ld, int nr,
                      DevStatus *st, uint64_t timeout_ns, int skip_if_converged) {
    if (skip_if_converged && converged(st)) return;
    const Ctx cx{rhs, ld, nr, st, timeout_ns, sd.backoff_ns, false, sd.n, sd.row_id, nullptr, 0};
    const int wpb = blockDim.x >> 5;
    const int32_t gw = blockIdx.x * wpb + (threadIdx.x >> 5);
    const int32_t nw = gridDim.x * wpb;
    prefetch_solve_inputs<T>(sd, rhs, sd.n, ld, nr);
    // every unknown of this launch starts as the "not computed" sentinel; one
    // grid barrier orders those stores before any poll
    {
        const int32_t gthreads = gridDim.x * blockDim.x;
        for (int32_t row = blockIdx.x * blockDim.x + threadIdx.x; row < sd.n; row += gthreads)
            for (int c = 0; c < nr; ++c)
                *reinterpret_cast<typename Bits<T>::U *>(out + (int64_t)row * ld + c) =
                    Sentinel<T>::bits;
    }
    if (!grid_barrier(st, gridDim.x, timeout_ns, -5)) {
        grid_exit(st);
        return;
    }
    // Chunks are taken in level order, each warp its own arithmetic sequence:
    // with every warp resident, the lowest unfinished chunk's warp has
    // finished its earlier chunks and all that chunk's dependencies lie in
    // earlier levels, so some warp can always make progress.
    // (Staging the next chunk's entries while this one waits measured slower
    // here than processing each chunk in turn: the staged loads compete with
    // the polls and pin registers; the barrier kernel keeps its staging.)
    const WarpChunks wc = warp_chunks(sd, gw, nw);
    int32_t c = wc.at(0);
    for (int32_t j = 1; c >= 0; ++j) {
        const int32_t cn = wc.at(j);   // in flight while this chunk runs
        if (process_chunk<T, L, R, true>(sd, c, out, cx)) break;
        c = cn;
    }
    grid_exit(st);
}

// ---------------------------------------------------------------------------
// Staged synchronisation-free solve, one right-hand side.
//
// Without staging a chunk issues, before its first gather, the load of its
// descriptor and then of its entries from HBM (measured on the 128^3 stencil
// at depth 2: 0.17 + 1.3 us ahead of a 0.7 us gather, per chunk).  Here each
// warp owns three shared-memory slots in a ring: while it solves the chunk in
// one, the next ones are copied in -- each chunk is stored once more as one
// contiguous blob (BlobLayout), so that the warp's 32 lanes bring it in with
// 16-byte asynchronous copies that complete on the slot's mbarrier -- and a
// chunk starts with all its gathers of x and b in flight at once, read from
// shared memory.  The copies of the chunk two ahead are issued right after
// this chunk's gathers, into the slot the previous chunk freed, so they
// overlap the gathers' latency.  (The bulk-copy engine was tried first: four
// small bulk copies per chunk cost 0.25-0.45 us to issue under load, and one
// engine per SM serialises 32 warps' requests.)
constexpr int kStageSlots = 3;
// per warp: the slots' headers (chunk, units; 16 bytes each) and mbarriers
// (8 bytes each), padded to 16 bytes, then the slots
constexpr int kStageHeadBytes = (kStageSlots * 24 + 15) & ~15;

// Units one slot holds: a chunk of 32 / L rows and z steps per lane.
template <typename T>
__host__ __device__ constexpr int stage_slot_units(int L, int z) {
    return BlobLayout<T>(32 / L, z, L).units;
}
template <typename T>
__host__ __device__ constexpr int stage_warp_bytes(int L, int z) {
    return kStageHeadBytes + kStageSlots * 16 * stage_slot_units<T>(L, z);
}

// The warp's slot ring (shared memory).
template <typename T>
struct StageRing {
    unsigned char *base;   // this warp's region
    int cap;               // units per slot
    __device__ __forceinline__ int4 *hdr(int sl) const {
        return reinterpret_cast<int4 *>(base) + sl;
    }
    __device__ __forceinline__ uint32_t bar(int sl) const {
        return smem_u32(base) + 16 * kStageSlots + 8 * sl;
    }
    __device__ __forceinline__ unsigned char *slot(int sl) const {
        return base + kStageHeadBytes + sl * 16 * cap;
    }
    // true if slot sl received (or is receiving) the chunk it holds
    __device__ __forceinline__ bool staged(int sl) const {
        const int4 h = *hdr(sl);
        return h.x >= 0 && h.y <= cap;
    }
    // All 32 lanes: slot sl takes chunk c (blob units [u0, u1)); copies are
    // started when it fits, and every lane arrives on the slot's barrier.
    __device__ __forceinline__ void fill(const SolveData<T> &sd, int sl, int32_t c, int64_t u0,
                                         int64_t u1) const {
        const int lane = threadIdx.x & 31;
        const int units = c >= 0 ? (int)(u1 - u0) : 0;
        if (lane == 0) *hdr(sl) = make_int4(c, units, 0, 0);
        if (c < 0 || units > cap) return;
        const uint32_t dst = smem_u32(slot(sl));
        const uint4 *src = sd.blob + u0;
        for (int u = lane; u < units; u += 32) cp_async16(dst + 16u * u, src + u);
        cp_async_mbar_arrive(bar(sl));
    }
};

// The refill of the ring that one chunk carries out once its gathers are in
// flight (or before an unstaged chunk): slot sl takes chunk c.
template <typename T>
struct Refill {
    const SolveData<T> &sd;
    StageRing<T> ring;
    int sl;
    int32_t c;
    int64_t u0, u1;
    __device__ __forceinline__ void operator()() const { ring.fill(sd, sl, c, u0, u1); }
};

// The L-bit mask of one row's lanes (from bit 0).
template <int L>
constexpr unsigned kGroupMask = L >= 32 ? 0xFFFFFFFFu : (1u << (L % 32)) - 1u;

// U steps of one lane's entries from the slot, gathered together: the terms
// already computed are summed into acc, the others are noted in `pend` (bit
// j0 + u) -- or, in a chunk wider than 32 steps (`defer` false: a slot holds
// a few long rows as well as many short ones), waited for on the spot.
// `hook` runs once the gathers are issued, if still pending (the ring's
// refill).
template <typename T, int U, typename Hook>
__device__ __forceinline__ void gather_steps(const int32_t *scol, const T *sval, int stride,
                                             int j0, bool defer, T *out, const Ctx &cx, T &acc,
                                             uint32_t &pend, bool &bail, const Hook &hook,
                                             bool &hook_pending) {
    int32_t cc[U];
    typename Bits<T>::U xb[U];
#pragma unroll
    for (int u = 0; u < U; ++u) cc[u] = scol[u * stride];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (cc[u] >= 0) xb[u] = Bits<T>::poll(out + (int64_t)cc[u] * cx.ld);
        else xb[u] = Bits<T>::of(other_term<T>(cx, cc[u], out, 0));
    }
    if (hook_pending) {
        hook();
        hook_pending = false;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (cc[u] >= 0 && xb[u] == Sentinel<T>::bits) {
            if (defer) pend |= 1u << (j0 + u);
            else acc = fma(-sval[u * stride],
                           wait_x<T>(out + (int64_t)cc[u] * cx.ld, cx.st, cx.timeout_ns,
                                     cx.backoff_ns, bail),
                           acc);
        } else {
            acc = fma(-sval[u * stride], Bits<T>::from(xb[u]), acc);
        }
    }
}

// Late terms of the warp's rows, each polled by the row's first lane: `gp`
// bit q = j * L + s stands for step j of lane s (entry j * stride + s from
// `scol`/`sval`, the row's own entries; 0 on every other lane).  The rounds
// are warp-wide, so that one FMA instruction serves every row with an
// arrival (on this GPU each FP64 instruction holds its pipe for many
// cycles, however few lanes it has): up to four terms per row are polled
// together per round, each arrival costs one dependent FMA, and a row is
// stored in the round its last term lands.
template <typename T, int L>
__device__ __forceinline__ void finish_late(const int32_t *scol, const T *sval, int stride,
                                            uint64_t gp, T *out, const Ctx &cx, T acc,
                                            bool scaled, const T *sdg, T *dst, bool &bail) {
    WaitBudget wb(cx.timeout_ns);
    unsigned it = 0;
    while (__any_sync(FULL_MASK, gp != 0)) {
        int bq[4];
        typename Bits<T>::U xb[4];
        uint64_t m = gp;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            bq[q] = m ? __ffsll((long long)m) - 1 : -1;
            m &= m - 1;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (bq[q] >= 0)
                xb[q] = Bits<T>::poll(out + (int64_t)scol[(bq[q] / L) * stride + bq[q] % L] * cx.ld);
        const bool had = gp != 0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (bq[q] >= 0 && xb[q] != Sentinel<T>::bits) {
                acc = fma(-sval[(bq[q] / L) * stride + bq[q] % L], Bits<T>::from(xb[q]), acc);
                gp &= ~(1ull << bq[q]);
            }
        if (had && gp == 0)
            store_x<T, true>(dst, scaled ? acc : div_by_diag<T>(acc, sdg[0], sdg[1]));
        if (gp && (++it & kPollMask) == 0 && wb.expired(cx.st, -2)) {
            bail = true;
            gp = 0;
        }
        if (cx.backoff_ns) __nanosleep(cx.backoff_ns);
    }
}

// Late terms when a row's pending set does not fit one 64-bit mask (L * z >
// 64): every lane polls its own, the late partial sums are reduced once more.
template <typename T, int L>
__device__ __forceinline__ void finish_late_lanes(const int32_t *scol, const T *sval, int stride,
                                                  uint32_t pend, T *out, const Ctx &cx, T &acc,
                                                  bool &bail) {
    T late = T(0);
    while (pend) {
        const int j = __ffs(pend) - 1;
        const T x = wait_x<T>(out + (int64_t)scol[j * stride] * cx.ld, cx.st, cx.timeout_ns,
                              cx.backoff_ns, bail);
        if (bail) break;
        late = fma(-sval[j * stride], x, late);
        pend &= pend - 1;
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) late += __shfl_xor_sync(FULL_MASK, late, o);
    acc += late;
}

// One staged chunk.  Every gather of every step is issued before anything is
// waited for; the lanes of a row reduce their early sums while the row still
// waits; the late terms are then polled by the row's first lane alone, so the
// row's last dependency is followed by one FMA and the store.  A blob marked
// scaled (descriptor .w != 0) holds the row's coefficients divided by its
// diagonal: its value starts as b_i / d_i (computed before any wait) and
// needs no division at the end.
template <typename T, int L>
__device__ __forceinline__ bool chunk_staged(const unsigned char *slot, T *out, const Ctx &cx,
                                             const Refill<T> &refill) {
    const int lane = threadIdx.x & 31;
    const int k = lane / L, s = lane % L;
    const int4 mt = *reinterpret_cast<const int4 *>(slot);
    const BlobLayout<T> lay(mt.y, mt.z, L);
    const bool active = k < mt.y;
    const bool scaled = mt.w != 0;
    // the row id and the diagonal stay in the slot (read again at the end)
    const int32_t *srow = reinterpret_cast<const int32_t *>(slot + 16 * lay.rows) + k;
    const T *sdg = reinterpret_cast<const T *>(slot + 16 * lay.diag) + 2 * k;
    T acc = T(0);
    bool bail = false;
    if (active && s == 0) {
        const T b = (T)load_rhs(cx, (int64_t)*srow * cx.ld);
        acc = scaled ? div_by_diag<T>(b, sdg[0], sdg[1]) : b;
    }
    const int stride = mt.y * L;
    const int32_t *rcol = reinterpret_cast<const int32_t *>(slot + 16 * lay.cols) + k * L;
    const T *rval = reinterpret_cast<const T *>(slot + 16 * lay.vals) + k * L;
    // every step of the row in as few batches as possible: batches of 5
    // (more spill at 64 registers), the remainder in one batch of its
    // exact size; the first batch issued carries the refill
    bool hook_pending = true;
    const bool defer = mt.z <= 32;
    uint32_t pend = 0;
    int j = 0;
    if (active)
        for (; j + 5 <= mt.z; j += 5)
            gather_steps<T, 5>(rcol + s + j * stride, rval + s + j * stride, stride, j, defer,
                               out, cx, acc, pend, bail, refill, hook_pending);
    switch (active ? mt.z - j : 0) {
#define SPTRSV_STEPS(UU)                                                                       \
    case UU:                                                                                   \
        gather_steps<T, UU>(rcol + s + j * stride, rval + s + j * stride, stride, j, defer,    \
                            out, cx, acc, pend, bail, refill, hook_pending);                   \
        break;
    SPTRSV_STEPS(1) SPTRSV_STEPS(2) SPTRSV_STEPS(3) SPTRSV_STEPS(4)
#undef SPTRSV_STEPS
    default: break;
    }
    if (hook_pending) refill();   // lanes without entries (inactive rows, empty rows)
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL_MASK, acc, o);
    const bool lead = active && s == 0;
    T *dst = out + (int64_t)(lead ? *srow : 0) * cx.ld;
    if (__any_sync(FULL_MASK, pend != 0)) {
        if (L * mt.z <= 64) {
            // the row's pending steps, lane by lane, gathered into its first
            // lane; rows with none are stored at once
            uint64_t gp = 0;
            for (int jj = 0; jj < mt.z; ++jj) {
                const unsigned bal = __ballot_sync(FULL_MASK, (pend >> jj) & 1u);
                const unsigned mine = (bal >> (k * L)) & kGroupMask<L>;
                gp |= (uint64_t)mine << (jj * L);
            }
            if (!lead) gp = 0;
            if (lead && gp == 0)
                store_x<T, true>(dst, scaled ? acc : div_by_diag<T>(acc, sdg[0], sdg[1]));
            finish_late<T, L>(rcol, rval, stride, gp, out, cx, acc, scaled, sdg, dst, bail);
            return __any_sync(FULL_MASK, bail);
        }
        finish_late_lanes<T, L>(rcol + s, rval + s, stride, active ? pend : 0u, out, cx, acc,
                                bail);
    }
    if (lead) store_x<T, true>(dst, scaled ? acc : div_by_diag<T>(acc, sdg[0], sdg[1]));
    return __any_sync(FULL_MASK, bail);
}

// Blob units [u0, u1) of chunk c (empty for c < 0).
template <typename T>
__device__ __forceinline__ void blob_range(const SolveData<T> &sd, int32_t c, int64_t &u0,
                                           int64_t &u1) {
    if (c < 0) {
        u0 = u1 = 0;
        return;
    }
    u0 = __ldg(sd.bofs + c);
    u1 = __ldg(sd.bofs + c + 1);
}

// Prologue of both staged kernels: the ring's barriers, and the copies of
// the warp's first two chunks into slots 0 and 1.
template <typename T>
__device__ __forceinline__ void ring_start(const SolveData<T> &sd, const StageRing<T> &ring,
                                           int32_t c0, int32_t c1) {
    if ((threadIdx.x & 31) == 0) {
        for (int sl = 0; sl < kStageSlots; ++sl) mbar_init(ring.bar(sl), 32);
        fence_mbar_init();
    }
    __syncwarp();
    int64_t u0, u1;
    blob_range(sd, c0, u0, u1);
    ring.fill(sd, 0, c0, u0, u1);
    blob_range(sd, c1, u0, u1);
    ring.fill(sd, 1, c1, u0, u1);
}

// After an abort: copies still in flight land before the CTA exits -- the
// current slot's (chunk c) if it was never seen complete, and those of the
// next two chunks cn1, cn2 (when their copies were started).
template <typename T>
__device__ __forceinline__ void ring_drain(const StageRing<T> &ring, int cur, int32_t c,
                                           int32_t cn1, int32_t cn2, bool cur_unwaited,
                                           uint32_t phase, uint64_t timeout_ns) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0 && c >= 0) {
        for (int k = 0; k < kStageSlots; ++k) {
            const int sl = (cur + k) % kStageSlots;
            const int32_t cs = k == 0 ? c : k == 1 ? cn1 : cn2;
            if (cs >= 0 && ring.staged(sl) && ring.hdr(sl)->x == cs && (k != 0 || cur_unwaited))
                mbar_drain(ring.bar(sl), (phase >> sl) & 1u, timeout_ns);
        }
    }
    __syncwarp();
}

// 88 registers: the gather batches and the late-term rounds fit without
// spilling, and five CTAs of 128 threads (or two of 256) stay resident per SM.
template <typename T, int L>
__global__ void __maxnreg__(88)
solve_staged_kernel(SolveData<T> sd, const double *rhs, T *out, int ld, DevStatus *st,
                    uint64_t timeout_ns, int skip_if_converged) {
    if (skip_if_converged && converged(st)) return;
    extern __shared__ __align__(128) unsigned char stage_smem[];
    const Ctx cx{rhs, ld, 1, st, timeout_ns, sd.backoff_ns, false, sd.n, sd.row_id, nullptr, 0};
    const int wpb = blockDim.x >> 5, wib = threadIdx.x >> 5;
    const int32_t gw = blockIdx.x * wpb + wib;
    const int32_t nw = gridDim.x * wpb;
    const StageRing<T> ring{stage_smem + (size_t)wib * stage_warp_bytes<T>(L, sd.stage_z),
                            stage_slot_units<T>(L, sd.stage_z)};
    const WarpChunks wc = warp_chunks(sd, gw, nw);
    // the warp's current chunk and the next two; the ring holds the current
    // one and the next, the chunk two ahead goes into the third slot while
    // the current one runs
    int32_t c = wc.at(0), cn1 = wc.at(1), cn2 = wc.at(2);
    ring_start(sd, ring, c, cn1);
    int64_t u2a, u2b;
    blob_range(sd, cn2, u2a, u2b);
    l2_prefetch_slice(sd.bofs, ((size_t)sd.nchunks + 1) * sizeof(int64_t));
    if (sd.n > 0) {
        size_t rb = ((size_t)(sd.n - 1) * ld + 1) * sizeof(double);
        if (rb > (64u << 20)) rb = 64u << 20;
        l2_prefetch_slice(rhs, rb);
    }
    // every unknown starts as the "not computed" sentinel; one grid barrier
    // orders those stores before any poll (the copies above fly meanwhile)
    {
        const int32_t gthreads = gridDim.x * blockDim.x;
        for (int32_t row = blockIdx.x * blockDim.x + threadIdx.x; row < sd.n; row += gthreads)
            *reinterpret_cast<typename Bits<T>::U *>(out + (int64_t)row * ld) = Sentinel<T>::bits;
    }
    const bool ok = grid_barrier(st, gridDim.x, timeout_ns, -5);
    if (sd.level_ns && blockIdx.x == 0 && threadIdx.x == 0) sd.level_ns[0] = globaltimer_ns();
    // Each warp solves its chunks in order (the progress argument of
    // solve_syncfree_kernel holds for both schedules; the copies a chunk
    // waits for depend on nothing but the structure).
    uint32_t phase = 0;   // bit s: parity of slot s's next completion
    int cur = 0;
    bool cur_unwaited = !ok;   // the current slot's copy was never seen complete
    if (!ok) cn2 = -1;         // the third slot was never filled
    for (int32_t j = 3; ok && c >= 0; ++j) {
        const int32_t cn3 = wc.at(j);   // in flight while this chunk runs
        const int nxt2 = cur == 0 ? 2 : cur - 1;   // (cur + 2) mod 3: the slot freed last
        const Refill<T> refill{sd, ring, nxt2, cn2, u2a, u2b};
        bool bail;
        if (ring.staged(cur)) {
            if (!__all_sync(FULL_MASK, mbar_wait(ring.bar(cur), (phase >> cur) & 1u, st,
                                                 timeout_ns, -6))) {
                cur_unwaited = true;
                cn2 = -1;   // its copies were not started
                break;
            }
            phase ^= 1u << cur;
            bail = chunk_staged<T, L>(ring.slot(cur), out, cx, refill);
        } else {
            refill();
            bail = chunk_one<T, L, true>(sd, c, out, cx);
        }
        if (bail) break;
        if (sd.level_ns && (threadIdx.x & 31) == 0)
            atomicMax(sd.level_ns + 1 + __ldg(sd.chunk_level + c),
                      (unsigned long long)globaltimer_ns());
        __syncwarp();
        blob_range(sd, cn3, u2a, u2b);
        c = cn1;
        cn1 = cn2;
        cn2 = cn3;
        cur = cur == kStageSlots - 1 ? 0 : cur + 1;
    }
    ring_drain(ring, cur, c, cn1, cn2, cur_unwaited, phase, timeout_ns);
    grid_exit(st);
}

template <typename T>
const void *pick_staged(int L) {
    switch (L) {
    case 1: return (const void *)solve_staged_kernel<T, 1>;
    case 2: return (const void *)solve_staged_kernel<T, 2>;
    case 4: return (const void *)solve_staged_kernel<T, 4>;
    case 8: return (const void *)solve_staged_kernel<T, 8>;
    case 16: return (const void *)solve_staged_kernel<T, 16>;
    case 32: return (const void *)solve_staged_kernel<T, 32>;
    }
    return nullptr;
}

template <typename T>
size_t stage_smem_bytes(int L, int stage_z, int block_threads) {
    return stage_z > 0 ? (size_t)(block_threads / 32) * stage_warp_bytes<T>(L, stage_z) : 0;
}




template <typename T, bool SF, int R>
const void *pick_l(int L) {
    if (R > 1) {
        return SF ? (const void *)solve_syncfree_kernel<T, 1, R>
                  : (const void *)solve_barrier_kernel<T, 1, R>;
    }
    switch (L) {
#define SPTRSV_CASE(LL)                                                        \
    case LL:                                                                   \
        return SF ? (const void *)solve_syncfree_kernel<T, LL, 1>              \
                  : (const void *)solve_barrier_kernel<T, LL, 1>;
        SPTRSV_CASE(1) SPTRSV_CASE(2) SPTRSV_CASE(4) SPTRSV_CASE(8) SPTRSV_CASE(16)
        SPTRSV_CASE(32)
#undef SPTRSV_CASE
    }
    return nullptr;
}

template <typename T, bool SF>
const void *pick(int L, int nr) {
    if (nr <= 1) return pick_l<T, SF, 1>(L);
    if (nr <= 2) return pick_l<T, SF, 2>(L);
    if (nr <= 4) return pick_l<T, SF, 4>(L);
    if (nr <= 8) return pick_l<T, SF, 8>(L);
    if (nr <= 16) return pick_l<T, SF, 16>(L);
    return pick_l<T, SF, 32>(L);
}

template <typename T>
const void *pick_kernel(int L, int nr, bool syncfree) {
    return syncfree ? pick<T, true>(L, nr) : pick<T, false>(L, nr);
}

// ---------------------------------------------------------------------------
// Refinement kernels (FP64 residual of the original L, FP32 corrections).

// r = b - A x with A the caller's operator.  The CSR holds the lower
// triangle the plan analysed; with rev it is P A P, so its row i is A's row
// n-1-i and its column c is A's column n-1-c.
__global__ void residual_kernel(int32_t n, const int32_t *__restrict__ row_ptr,
                                const int32_t *__restrict__ col,
                                const double *__restrict__ val, int rev,
                                const double *__restrict__ b, const double *__restrict__ x,
                                double *__restrict__ r, int nr, int ld, DevStatus *st) {
    if (converged(st)) return;
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    double rmax = 0.0, xmax = 0.0;
    if (i < n) {
        const int32_t a = row_ptr[i], e = row_ptr[i + 1];
        const int64_t ri = rev ? n - 1 - i : i;
        for (int c = 0; c < nr; ++c) {
            double s = b[ri * ld + c];
            for (int32_t k = a; k < e; ++k) {
                const int64_t j = rev ? n - 1 - col[k] : col[k];
                s -= val[k] * x[j * ld + c];
            }
            r[ri * ld + c] = s;
            rmax = fmax(rmax, fabs(s));
            xmax = fmax(xmax, fabs(x[ri * ld + c]));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rmax = fmax(rmax, __shfl_xor_sync(FULL_MASK, rmax, o));
        xmax = fmax(xmax, __shfl_xor_sync(FULL_MASK, xmax, o));
    }
    if ((threadIdx.x & 31) == 0) {
        unsigned long long *nm = reinterpret_cast<unsigned long long *>(st->norms);
        atomicMax(&nm[0], (unsigned long long)__double_as_longlong(rmax));
        atomicMax(&nm[1], (unsigned long long)__double_as_longlong(xmax));
    }
}

__global__ void ir_bnorm_kernel(DevStatus *st, const double *__restrict__ b, int64_t count) {
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(b[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(FULL_MASK, m, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(reinterpret_cast<unsigned long long *>(&st->norms[2]),
                  (unsigned long long)__double_as_longlong(m));
}

__global__ void ir_decide_kernel(DevStatus *st, double tol, const unsigned long long *lnorm) {
    unsigned long long *nm = reinterpret_cast<unsigned long long *>(st->norms);
    if (st->ir_flag) return;
    const double rn = __longlong_as_double((long long)nm[0]);
    const double xn = __longlong_as_double((long long)nm[1]);
    const double bn = __longlong_as_double((long long)nm[2]);
    const double ln = __longlong_as_double((long long)*lnorm);
    if (rn <= tol * (ln * xn + bn)) st->ir_flag = 1ull;
    else st->ir_iters += 1;
    nm[0] = 0ull;
    nm[1] = 0ull;
}

__global__ void ir_update_kernel(double *__restrict__ x, const float *__restrict__ d,
                                 int64_t count, int first, DevStatus *st) {
    if (!first && converged(st)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    x[i] = first ? (double)d[i] : x[i] + (double)d[i];
}


// ---------------------------------------------------------------------------
// Batched persistent solve.

__device__ __forceinline__ bool group_barrier(unsigned long long *cnt, unsigned long long target,
                                              DevStatus *st, uint64_t timeout_ns) {
    __shared__ int s_gok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        red_release_add_u64(cnt, 1ull);
        if (ld_acquire_u64(cnt) < target) {
            WaitBudget wb(timeout_ns);
            unsigned it = 0;
            while (ld_acquire_u64(cnt) < target) {
                if ((++it & kPollMask) == 0 && wb.expired(st, -3)) { ok = 0; break; }
            }
        }
        s_gok = ok;
    }
    __syncthreads();
    return s_gok != 0;
}

template <typename T>
__device__ __forceinline__ bool batch_chunk(const SolveData<T> &sd, int32_t c, T *out,
                                            const Ctx &cx, int R) {
    switch (R) {
    case 1:  // one right-hand side: the lanes-per-row chunk processor
        switch (sd.L) {
        case 1: return chunk_one<T, 1, true>(sd, c, out, cx);
        case 2: return chunk_one<T, 2, true>(sd, c, out, cx);
        case 4: return chunk_one<T, 4, true>(sd, c, out, cx);
        case 8: return chunk_one<T, 8, true>(sd, c, out, cx);
        case 16: return chunk_one<T, 16, true>(sd, c, out, cx);
        default: return chunk_one<T, 32, true>(sd, c, out, cx);
        }
    case 2: return chunk_multi<T, 2, true>(sd, c, out, cx);
    case 4: return chunk_multi<T, 4, true>(sd, c, out, cx);
    case 8: return chunk_multi<T, 8, true>(sd, c, out, cx);
    case 16: return chunk_multi<T, 16, true>(sd, c, out, cx);
    default: return chunk_multi<T, 32, true>(sd, c, out, cx);
    }
}

// sync-free solve of one matrix by the warps of its group; false on abort
template <typename T>
__device__ __forceinline__ bool batch_solve_group(const SolveData<T> &sd, const double *rhs,
                                                  bool rhs_coherent, T *out, int nr, int R,
                                                  DevStatus *st, uint64_t timeout_ns, int32_t gw,
                                                  int32_t nw) {
    const Ctx cx{rhs, nr, nr, st, timeout_ns, 0, rhs_coherent, sd.n, sd.row_id, nullptr, 0};
    for (int32_t c = gw; c < sd.nchunks; c += nw)
        if (batch_chunk<T>(sd, c, out, cx, R)) return false;
    return true;
}

__device__ __forceinline__ void atomic_max_abs(unsigned long long *slot, double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL_MASK, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(slot, (unsigned long long)__double_as_longlong(v));
}

// One matrix's part of the batched solve, run by the CTAs of its group
// (j-th of G); returns early (every thread of the CTA alike) on an abort.
template <bool IR>
__device__ __forceinline__ void batch_group(const BatchMat &M, BatchCtl *C, DevStatus *st,
                                            double tol, int max_iter, uint64_t timeout_ns,
                                            int32_t j, int32_t G) {
    const int wpb = blockDim.x >> 5;
    const int32_t gw = j * wpb + (threadIdx.x >> 5), nw = G * wpb;
    const int64_t gt = (int64_t)j * blockDim.x + threadIdx.x, gthreads = (int64_t)G * blockDim.x;
    const int64_t count = (int64_t)M.n * M.nr;
    unsigned long long bar = 0;
#define SPTRSV_GSYNC()                                                               \
    if (!group_barrier(&C->bar, (++bar) * (unsigned long long)G, st, timeout_ns)) return
    if (!IR) {
        for (int64_t i = gt; i < count; i += gthreads)
            *reinterpret_cast<unsigned long long *>(M.x + i) = Sentinel<double>::bits;
        SPTRSV_GSYNC();
        batch_solve_group<double>(M.s64, M.b, false, M.x, M.nr, M.R, st, timeout_ns, gw, nw);
        return;
    }
    // FP32 solve, then FP64 residual / FP32 correction rounds
    double bmax = 0.0;
    for (int64_t i = gt; i < count; i += gthreads) {
        *reinterpret_cast<unsigned *>(M.d32 + i) = Sentinel<float>::bits;
        bmax = fmax(bmax, fabs(M.b[i]));
    }
    atomic_max_abs(&C->norms[0][2], bmax);
    SPTRSV_GSYNC();
    if (!batch_solve_group<float>(M.s32, M.b, false, M.d32, M.nr, M.R, st, timeout_ns, gw, nw)) return;
    SPTRSV_GSYNC();
    // values written by other CTAs of the group are read through L2 (__ldcg):
    // this SM's L1 may hold stale copies of those lines
    for (int64_t i = gt; i < count; i += gthreads) M.x[i] = (double)__ldcg(M.d32 + i);
    int it = 0;
    for (; it < max_iter; ++it) {
        SPTRSV_GSYNC();
        // r = b - L x and the infinity norms of r and x
        double rmax = 0.0, xmax = 0.0;
        for (int64_t row = gt; row < (int64_t)M.n; row += gthreads) {
            const int32_t a = M.row_ptr[row], e = M.row_ptr[row + 1];
            const int64_t ri = M.rev ? M.n - 1 - row : row;  // see residual_kernel
            for (int c = 0; c < M.nr; ++c) {
                double s = M.b[ri * M.nr + c];
                for (int32_t k = a; k < e; ++k) {
                    const int64_t j = M.rev ? M.n - 1 - M.col[k] : M.col[k];
                    s -= M.val[k] * __ldcg(M.x + j * M.nr + c);
                }
                M.r64[ri * M.nr + c] = s;
                rmax = fmax(rmax, fabs(s));
                xmax = fmax(xmax, fabs(__ldcg(M.x + ri * M.nr + c)));
            }
        }
        atomic_max_abs(&C->norms[it][0], rmax);
        atomic_max_abs(&C->norms[it][1], xmax);
        SPTRSV_GSYNC();
        const double rn = __longlong_as_double((long long)ld_relaxed_u64(&C->norms[it][0]));
        const double xn = __longlong_as_double((long long)ld_relaxed_u64(&C->norms[it][1]));
        const double bnorm = __longlong_as_double((long long)ld_relaxed_u64(&C->norms[0][2]));
        if (rn <= tol * (M.lnorm * xn + bnorm)) break;
        for (int64_t i = gt; i < count; i += gthreads)
            *reinterpret_cast<unsigned *>(M.d32 + i) = Sentinel<float>::bits;
        SPTRSV_GSYNC();
        if (!batch_solve_group<float>(M.s32, M.r64, true, M.d32, M.nr, M.R, st, timeout_ns, gw, nw))
            return;
        SPTRSV_GSYNC();
        for (int64_t i = gt; i < count; i += gthreads)
            M.x[i] = __ldcg(M.x + i) + (double)__ldcg(M.d32 + i);
    }
    if (gt == 0) {
        C->iters = it;
        C->converged = it < max_iter ? 1 : 0;
    }
#undef SPTRSV_GSYNC
}

template <bool IR>
__global__ void __launch_bounds__(kMaxSolveThreads)
batch_kernel(const BatchMat *__restrict__ mats, int32_t nmats, BatchCtl *ctl, DevStatus *st,
             double tol, int max_iter, uint64_t timeout_ns) {
    __shared__ int32_t s_m;
    if (threadIdx.x == 0) {
        int32_t lo = 0, hi = nmats - 1;
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (mats[mid].cta_begin <= (int32_t)blockIdx.x) lo = mid; else hi = mid - 1;
        }
        s_m = lo;
    }
    __syncthreads();
    const BatchMat &M = mats[s_m];
    const int32_t j = (int32_t)blockIdx.x - M.cta_begin;
    const int32_t G = M.cta_count;
    if (j < 0 || j >= G || M.n == 0) return;
    BatchCtl *C = ctl + s_m;
    if (threadIdx.x == 0) atomicCAS(&C->t_begin, 0ull, (unsigned long long)globaltimer_ns());
    batch_group<IR>(M, C, st, tol, max_iter, timeout_ns, j, G);
    if (threadIdx.x == 0) atomicMax(&C->t_end, (unsigned long long)globaltimer_ns());
}
}  // namespace

// ---------------------------------------------------------------------------
// Chunk blobs (BlobLayout) of a solve structure.
namespace {
template <typename T>
__global__ void blob_units_kernel(int32_t nchunks, int L, const int4 *__restrict__ meta,
                                  int64_t *units) {
    const int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nchunks) return;
    const int4 m = meta[c];
    units[c] = BlobLayout<T>(m.y, m.z, L).units;
}

template <typename T> struct MinNormal;
template <> struct MinNormal<double> { static constexpr double v = 2.2250738585072014e-308; };
template <> struct MinNormal<float> { static constexpr float v = 1.17549435e-38f; };

// one warp per chunk; the blob array is zeroed beforehand (padding).  The
// chunk's coefficients are stored divided by their row's diagonal (IEEE
// division) and the descriptor's .w set to 1, unless a quotient of a
// non-zero coefficient would leave the normal range (overflow, underflow,
// a zero, infinite or NaN diagonal, a non-finite coefficient): then the
// chunk keeps its coefficients as they are (.w = 0) and the kernel divides
// at the end.
template <typename T>
__global__ void blob_fill_kernel(int32_t nchunks, int L, const int4 *__restrict__ meta,
                                 const int32_t *__restrict__ row_id, const T *__restrict__ diag,
                                 const int32_t *__restrict__ ecol, const T *__restrict__ eval,
                                 const int64_t *__restrict__ bofs, uint4 *blob) {
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= nchunks) return;
    const int4 m = meta[c];
    const BlobLayout<T> lay(m.y, m.z, L);
    unsigned char *base = reinterpret_cast<unsigned char *>(blob + bofs[c]);
    int32_t *rows = reinterpret_cast<int32_t *>(base + 16 * lay.rows);
    T *dg = reinterpret_cast<T *>(base + 16 * lay.diag);
    int32_t *cols = reinterpret_cast<int32_t *>(base + 16 * lay.cols);
    T *vals = reinterpret_cast<T *>(base + 16 * lay.vals);
    for (int k = lane; k < m.y; k += 32) rows[k] = row_id[m.x + k];
    for (int e = lane; e < 2 * m.y; e += 32) dg[e] = diag[2 * (int64_t)m.x + e];
    const int ne = m.z * m.y * L;
    const int per_step = m.y * L;
    bool ok = true;
    for (int e = lane; e < ne; e += 32) {
        const T v = eval[(int64_t)m.w + e];
        if (v == T(0)) continue;
        const T d = diag[2 * ((int64_t)m.x + (e % per_step) / L)];
        const T q = v / d;
        ok = ok && isfinite(q) && fabs(q) >= MinNormal<T>::v;
    }
    const bool scaled = __all_sync(0xFFFFFFFFu, ok);
    for (int e = lane; e < ne; e += 32) {
        cols[e] = ecol[(int64_t)m.w + e];
        const T v = eval[(int64_t)m.w + e];
        vals[e] = scaled ? v / diag[2 * ((int64_t)m.x + (e % per_step) / L)] : v;
    }
    if (lane == 0) *reinterpret_cast<int4 *>(base) = make_int4(m.x, m.y, m.z, scaled ? 1 : 0);
}
}  // namespace

template <typename T>
cudaError_t launch_blob_units(int32_t nchunks, int L, const int4 *meta, int64_t *units,
                              cudaStream_t s) {
    if (nchunks <= 0) return cudaSuccess;
    blob_units_kernel<T><<<(nchunks + 255) / 256, 256, 0, s>>>(nchunks, L, meta, units);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_blob_fill(int32_t nchunks, int L, const int4 *meta, const int32_t *row_id,
                             const T *diag, const int32_t *ecol, const T *eval,
                             const int64_t *bofs, uint4 *blob, cudaStream_t s) {
    if (nchunks <= 0) return cudaSuccess;
    const int64_t threads = (int64_t)nchunks * 32;
    blob_fill_kernel<T><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        nchunks, L, meta, row_id, diag, ecol, eval, bofs, blob);
    return cudaGetLastError();
}
template cudaError_t launch_blob_units<double>(int32_t, int, const int4 *, int64_t *,
                                               cudaStream_t);
template cudaError_t launch_blob_units<float>(int32_t, int, const int4 *, int64_t *,
                                              cudaStream_t);
template cudaError_t launch_blob_fill<double>(int32_t, int, const int4 *, const int32_t *,
                                              const double *, const int32_t *, const double *,
                                              const int64_t *, uint4 *, cudaStream_t);
template cudaError_t launch_blob_fill<float>(int32_t, int, const int4 *, const int32_t *,
                                             const float *, const int32_t *, const float *,
                                             const int64_t *, uint4 *, cudaStream_t);

template <typename T>
int stage_cap_z(int L, int smem_per_sm, int warps) {
    int z = 0;
    // 1 KiB reserved per CTA: up to 8 CTAs (blocks of 128 threads) per SM
    const int budget = smem_per_sm - 8 * 1024;
    for (int c = 1; c <= kStageZMax; ++c)
        if (warps * stage_warp_bytes<T>(L, c) <= budget) z = c;
    return z;
}
template int stage_cap_z<double>(int, int, int);
template int stage_cap_z<float>(int, int, int);

int batch_max_coresident(bool ir, int block_threads, int num_sms) {
    int per_sm = 0;
    const void *k = ir ? (const void *)batch_kernel<true> : (const void *)batch_kernel<false>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block_threads, 0) != cudaSuccess)
        return 0;
    return per_sm * num_sms;
}

cudaError_t launch_batch(const BatchMat *mats, int32_t nmats, BatchCtl *ctl, DevStatus *st,
                         bool ir, double tol, int max_iter, uint64_t timeout_ns, int block_threads,
                         int grid, cudaStream_t s) {
    if (nmats == 0 || grid == 0) return cudaSuccess;
    if (max_iter > kBatchMaxIter) max_iter = kBatchMaxIter;
    void *args[] = {(void *)&mats, (void *)&nmats, (void *)&ctl, (void *)&st,
                    (void *)&tol, (void *)&max_iter, (void *)&timeout_ns};
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(grid);
    lc.blockDim = dim3(block_threads);
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    const void *k = ir ? (const void *)batch_kernel<true> : (const void *)batch_kernel<false>;
    return cudaLaunchKernelExC(&lc, k, args);
}

template <typename T>
size_t run_smem_bytes(int nr, bool syncfree, int run_slots) {
    return (!syncfree && nr <= 1 && run_slots > 0) ? (size_t)run_slots * sizeof(T) : 0;
}

// The kernel a launch runs, its block size and dynamic shared memory.
struct KernelPick {
    const void *k;
    int block;
    size_t smem;
};
template <typename T>
KernelPick choose_kernel(int L, int nr, bool syncfree, int block_threads, int run_slots,
                         int stage_z) {
    const int bt = block_threads < kMaxSolveThreads ? block_threads : kMaxSolveThreads;
    if (syncfree && nr <= 1 && stage_z > 0)
        return {pick_staged<T>(L), bt, stage_smem_bytes<T>(L, stage_z, bt)};
    return {pick_kernel<T>(L, nr, syncfree), bt, run_smem_bytes<T>(nr, syncfree, run_slots)};
}

template <typename T>
int max_coresident_ctas(int L, int nr, bool syncfree, int block_threads, int num_sms,
                        int run_slots, int stage_z) {
    const KernelPick kp = choose_kernel<T>(L, nr, syncfree, block_threads, run_slots, stage_z);
    if (!kp.k) return 0;
    if (kp.smem > 48 * 1024 &&
        cudaFuncSetAttribute(kp.k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kp.smem) !=
            cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kp.k, kp.block, kp.smem) !=
        cudaSuccess)
        return 0;
    return per_sm * num_sms;
}
template int max_coresident_ctas<double>(int, int, bool, int, int, int, int);
template int max_coresident_ctas<float>(int, int, bool, int, int, int, int);

template <typename T>
cudaError_t launch_solve(const SolveData<T> &sd, const double *rhs, T *out, int32_t n,
                         int ld, int nr, bool syncfree, const LaunchCfg &cfg,
                         DevStatus *st, uint64_t timeout_ns, bool skip_if_converged,
                         cudaStream_t s) {
    if (n == 0 || nr == 0) return cudaSuccess;
    if (sd.stage_z < 0 || sd.stage_z > kStageZMax) return cudaErrorInvalidValue;
    SolveData<T> sdc = sd;
    if (!sdc.blob || !sdc.bofs) sdc.stage_z = 0;   // no blobs: the unstaged kernels
    const KernelPick kp = choose_kernel<T>(sdc.L, nr, syncfree, cfg.block_threads,
                                           sdc.run_slots, sdc.stage_z);
    const bool staged = syncfree && nr == 1 && sdc.stage_z > 0;
    const void *k = kp.k;
    if (!k) return cudaErrorInvalidValue;
    const int skip = skip_if_converged ? 1 : 0;
    void *args[] = {(void *)&sdc, (void *)&rhs,        (void *)&out,  (void *)&ld,
                    (void *)&nr,  (void *)&st,         (void *)&timeout_ns,
                    (void *)&skip};
    void *sargs[] = {(void *)&sdc, (void *)&rhs, (void *)&out, (void *)&ld,
                     (void *)&st,  (void *)&timeout_ns, (void *)&skip};
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(cfg.grid);
    lc.blockDim = dim3(kp.block);
    lc.dynamicSmemBytes = kp.smem;
    if (lc.dynamicSmemBytes > 48 * 1024) {
        cudaError_t ea = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)lc.dynamicSmemBytes);
        if (ea != cudaSuccess) return ea;
    }
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    return cudaLaunchKernelExC(&lc, k, staged ? sargs : args);
}
template cudaError_t launch_solve<double>(const SolveData<double> &, const double *, double *,
                                          int32_t, int, int, bool, const LaunchCfg &,
                                          DevStatus *, uint64_t, bool, cudaStream_t);
template cudaError_t launch_solve<float>(const SolveData<float> &, const double *, float *,
                                         int32_t, int, int, bool, const LaunchCfg &,
                                         DevStatus *, uint64_t, bool, cudaStream_t);

cudaError_t launch_residual(int32_t n, const int32_t *row_ptr, const int32_t *col,
                            const double *val, bool rev, const double *b, const double *x,
                            double *r, int nr, int ld, DevStatus *st, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    residual_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, row_ptr, col, val, rev ? 1 : 0, b, x, r,
                                                    nr, ld, st);
    return cudaGetLastError();
}

cudaError_t launch_ir_begin(DevStatus *st, const double *b, int64_t count, cudaStream_t s) {
    // reset ir_iters (int at offset 12) and ir_flag + norms
    cudaError_t e = cudaMemsetAsync(&st->ir_iters, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(&st->ir_flag, 0, sizeof(unsigned long long) + sizeof(st->norms), s);
    if (e != cudaSuccess) return e;
    if (count > 0) {
        int64_t blocks = (count + 255) / 256;
        if (blocks > 4096) blocks = 4096;
        ir_bnorm_kernel<<<(unsigned)blocks, 256, 0, s>>>(st, b, count);
    }
    return cudaGetLastError();
}

cudaError_t launch_ir_decide(DevStatus *st, double tol, const unsigned long long *lnorm,
                             cudaStream_t s) {
    ir_decide_kernel<<<1, 1, 0, s>>>(st, tol, lnorm);
    return cudaGetLastError();
}

cudaError_t launch_ir_update(double *x, const float *d, int64_t count, bool first,
                             DevStatus *st, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    ir_update_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(x, d, count, first ? 1 : 0,
                                                                    st);
    return cudaGetLastError();
}

}  // namespace sptrsv
