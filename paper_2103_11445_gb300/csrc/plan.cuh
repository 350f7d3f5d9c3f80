// Host-side plan object shared by the C entry points (api.cu) and the
// batched solve (batch.cu).
#pragma once

#include <cstring>
#include <vector>

#include "solve.cuh"
#include "transform.cuh"

namespace sptrsv {

// Owning device array (cudaMalloc / cudaFree).
template <typename T>
struct DevArr {
    T *p = nullptr;
    size_t n = 0;
    DevArr() = default;
    DevArr(const DevArr &) = delete;
    DevArr &operator=(const DevArr &) = delete;
    DevArr(DevArr &&o) noexcept { swap(o); }
    DevArr &operator=(DevArr &&o) noexcept {
        if (this != &o) {
            reset();
            swap(o);
        }
        return *this;
    }
    ~DevArr() { reset(); }
    void reset() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    cudaError_t alloc(size_t count) {
        reset();
        if (count == 0) return cudaSuccess;
        cudaError_t e = cudaMalloc((void **)&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        n = count;
        return cudaSuccess;
    }
    void swap(DevArr &o) {
        std::swap(p, o.p);
        std::swap(n, o.n);
    }
};

template <typename T>
struct SolveStruct {
    DevArr<int32_t> lvl_chunk, ecol, row_id, chunk_level;
    DevArr<int4> meta;
    DevArr<T> eval, diag;
    DevArr<int2> phases;
    int32_t n = 0, nlev = 0, nchunks = 0, L = 1, nphases = 0;
    int32_t run_slots = 0;      // rows of the largest CTA-local run (shared memory)
    DevArr<int32_t> chunk_run_p0;  // first position of the chunk's run, -1 outside runs
    int32_t run_encoded = -1;   // run threshold the entries are encoded for (-1: none)
    int64_t nslots = 0;
    int32_t width_p99 = 0;      // steps per lane covering 99% of the chunks
    std::vector<int32_t> h_lvl_chunk;  // host copy of lvl_chunk
    DevArr<int32_t> sched, sched_ptr;  // level-major chunk schedule (SolveData)
    int32_t sched_nw = 0;              // warps it was dealt to (0: none)
    DevArr<uint4> blob;                // chunk blobs of the staged kernels
    DevArr<int64_t> bofs;              // [nchunks + 1] unit offsets into blob
    bool blob_valid = false;           // blob matches the current entries
    bool built = false;
    SolveData<T> view() const {
        SolveData<T> v;
        v.n = n;
        v.nlev = nlev;
        v.nchunks = nchunks;
        v.L = L;
        v.lvl_chunk = lvl_chunk.p;
        v.meta = meta.p;
        v.ecol = ecol.p;
        v.eval = eval.p;
        v.row_id = row_id.p;
        v.diag = diag.p;
        v.phases = phases.p;
        v.nphases = nphases;
        v.backoff_ns = 0;
        v.run_slots = run_slots;
        v.stage_z = 0;          // set per launch (stage_width)
        v.sched = sched.p;
        v.sched_ptr = sched_ptr.p;
        v.sched_nw = sched.p ? sched_nw : 0;
        v.blob = blob_valid ? blob.p : nullptr;
        v.bofs = blob_valid ? bofs.p : nullptr;
        v.chunk_level = chunk_level.p;
        v.level_ns = nullptr;   // set by a level-timed solve
        return v;
    }
};

// Records of the single-CTA tail (see TailData in solve.cuh).
// A kernel generated for one tail segment (the runtime compiler's output,
// loaded as a library; unloaded with its owner).
struct GenKernel {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t fn = nullptr;
    size_t smem = 0;
    GenKernel() = default;
    GenKernel(const GenKernel &) = delete;
    GenKernel &operator=(const GenKernel &) = delete;
    GenKernel(GenKernel &&o) noexcept { swap(o); }
    GenKernel &operator=(GenKernel &&o) noexcept {
        if (this != &o) {
            reset();
            swap(o);
        }
        return *this;
    }
    ~GenKernel() { reset(); }
    void reset() {
        if (lib) cudaLibraryUnload(lib);
        lib = nullptr;
        fn = nullptr;
        smem = 0;
    }
    void swap(GenKernel &o) {
        std::swap(lib, o.lib);
        std::swap(fn, o.fn);
        std::swap(smem, o.smem);
    }
};

struct TailSeg {
    int32_t lev0 = 0;        // first new level of the segment
    int32_t c0 = 0;          // its first chunk
    int32_t P0 = 0;          // its first solve position
    int32_t nrows = 0, nlev = 0, K = 0, T = 0, W = 0;
    DevArr<int32_t> lp, row, nn, acol;
    DevArr<int4> term;
    DevArr<double2> diag;
    DevArr<double> aval, s0;
    DevArr<int64_t> aptr;
    GenKernel gen;           // generated kernel of the segment (fn null: none)
};

struct TailStruct {
    int32_t for_rows = 0;    // width limit the records were built for
    int32_t lev0 = 0;        // first new level of the tail (its first segment's)
    int32_t c0 = 0;          // its first chunk
    int32_t nlev = 0;        // levels of all segments (0: no tail)
    std::vector<TailSeg> segs;   // in solve order
    bool built = false;
    int32_t gen_rows = 0;    // codegen_rows the generated kernels were made for
    double gen_ms = 0;       // time spent generating and compiling them
};

struct SolveConfig {
    bool syncfree = false;
    int L = 1;
    int block_threads = 512;
    int grid = 0;
    int tail_rows = 0;      // single-CTA tail over trailing levels of at most this
                            // many rows (0: none)
    int cta_run_rows = 0;   // resolved threshold (<= 0: no runs)
    int backoff_ns = 0;     // synchronisation-free polling back-off
    bool stage_off = false; // synchronisation-free solve without shared-memory staging
    bool sched_lm = false;  // synchronisation-free chunks dealt level-major (else round robin)
};

}  // namespace sptrsv

struct sptrsv_plan_s {
    int device = 0;
    int num_sms = 0;
    int smem_per_sm = 0;         // shared memory of one SM (bytes)
    int32_t n = 0;
    int64_t nnz = 0;
    int32_t op = 0;              // SPTRSV_OP_* the caller asked for
    bool rev = false;            // row_ptr/col/val hold P A P (A upper): the
                                 // solve structure is mirrored back to A's numbering
    sptrsv::DevArr<int32_t> row_ptr, col;   // the lower-triangular operator analysed
    sptrsv::DevArr<double> val;
    sptrsv::DevArr<int32_t> offdeg, level, level_ptr, perm;
    std::vector<int32_t> h_level_ptr;
    int32_t nlev = 0;
    int64_t offdeg_hist[4] = {0, 0, 0, 0};   // rows with 0 | 1-2 | 3-6 | >= 7 dependencies
    sptrsv::DevArr<sptrsv::DevStatus> status;
    sptrsv::DevArr<unsigned long long> lnorm;
    // transform
    std::vector<int32_t> seg_first, seg_depth;
    sptrsv::DevArr<int64_t> rw_off;
    sptrsv::DevArr<int32_t> rw_col, rw_nb, pos_item;
    sptrsv::DevArr<double> rw_val;
    int64_t nitems = 0;
    int64_t nnz_x = 0, nnz_b = 0;
    int32_t rows_rewritten = 0;
    sptrsv::SolveStruct<double> s64;
    sptrsv::TailStruct tail;              // of s64 (FP64, one right-hand side)
    sptrsv::SolveStruct<float> s32;
    sptrsv_transform_params_t prm{};
    sptrsv::SolveConfig cfg;
    // refinement buffers
    sptrsv::DevArr<float> d32;
    sptrsv::DevArr<double> r64;
    double analyze_ms = 0.0, transform_ms = 0.0;
    int32_t thin_rows_used = 0;
    sptrsv_status_t latched = SPTRSV_OK;
    sptrsv_mlp_t costmodel = nullptr;  // not owned
    int32_t chosen_depth = -1;         // depth picked by the cost model (-1: none)
    bool tuned_from_cache = false;     // the last autotuning reused a cached launch
    bool injected = false;             // sptrsv_debug_inject_wait was applied: no tail
    // profiling: events around the main solve kernel of the last solve
    bool profiling = false;
    cudaEvent_t prof_ev[2] = {nullptr, nullptr};
    bool prof_valid = false;
    ~sptrsv_plan_s() {
        if (prof_ev[0]) cudaEventDestroy(prof_ev[0]);
        if (prof_ev[1]) cudaEventDestroy(prof_ev[1]);
    }
};
