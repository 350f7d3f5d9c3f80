// Per-matrix generated kernels for thin tail segments: the GPU form of the
// paper's specialised code generation (Sec. IV, Fig. 4: one piece of code
// per level with the matrix's indices and values written in as constants,
// indirect indexing gone from the rewritten rows).
//
// On a SIMT GPU a level whose rows take different code paths serialises
// them within a warp, so generated code pays only where a level holds about
// one row -- the thin, nearly serial segments the rewriting targets (chains,
// two-row levels).  There one thread runs the segment's rows in solve order
// (a valid topological order), with no barrier between levels: each row is
// its folded constant (the fold pass of the tail) plus one FMA per
// in-segment term, the coefficient an immediate, the unknown read from a
// register when the same generated function solved it (32 rows each) and
// from shared memory otherwise.  The source is compiled at transform time by the runtime
// compiler (NVRTC, loaded on demand) straight to a cubin for this GPU, which
// the CUDA runtime loads as a library; nothing reads the compiled code.
#include <dlfcn.h>
#include <nvrtc.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "codegen.cuh"

namespace sptrsv {
namespace {

// The runtime compiler's entry points, resolved from the shared library at
// first use (the library does not link against it).
struct NvrtcApi {
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
    bool ok = false;
};

NvrtcApi &nvrtc() {
    static NvrtcApi api;
    static std::once_flag once;
    std::call_once(once, [] {
        std::vector<std::string> names = {"libnvrtc.so.13", "libnvrtc.so"};
        if (const char *home = std::getenv("CUDA_HOME")) {
            names.push_back(std::string(home) + "/lib64/libnvrtc.so.13");
            names.push_back(std::string(home) + "/lib64/libnvrtc.so");
        }
        names.push_back("/usr/local/cuda/lib64/libnvrtc.so.13");
        names.push_back("/usr/local/cuda/lib64/libnvrtc.so");
        void *h = nullptr;
        for (const std::string &n : names)
            if ((h = dlopen(n.c_str(), RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
        if (!h) return;
        api.create = reinterpret_cast<decltype(api.create)>(dlsym(h, "nvrtcCreateProgram"));
        api.compile = reinterpret_cast<decltype(api.compile)>(dlsym(h, "nvrtcCompileProgram"));
        api.cubin_size = reinterpret_cast<decltype(api.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
        api.cubin = reinterpret_cast<decltype(api.cubin)>(dlsym(h, "nvrtcGetCUBIN"));
        api.log_size =
            reinterpret_cast<decltype(api.log_size)>(dlsym(h, "nvrtcGetProgramLogSize"));
        api.log = reinterpret_cast<decltype(api.log)>(dlsym(h, "nvrtcGetProgramLog"));
        api.destroy = reinterpret_cast<decltype(api.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
        api.ok = api.create && api.compile && api.cubin_size && api.cubin && api.log_size &&
                 api.log && api.destroy;
    });
    return api;
}

// A double as a C++ literal that reads back to the same bits.
std::string literal(double v) {
    char b[64];
    if (std::isfinite(v)) {
        std::snprintf(b, sizeof b, "%a", v);
    } else {
        unsigned long long u;
        std::memcpy(&u, &v, sizeof u);
        std::snprintf(b, sizeof b, "__longlong_as_double(0x%llxULL)", u);
    }
    return b;
}

double from_halves(int lo, int hi) {
    const unsigned long long u =
        ((unsigned long long)(unsigned)hi << 32) | (unsigned long long)(unsigned)lo;
    double v;
    std::memcpy(&v, &u, sizeof v);
    return v;
}

constexpr int32_t kRowsPerFn = 32;   // rows per generated function

}  // namespace

const char *codegen_entry_name() { return "sptrsv_gen_segment"; }

bool codegen_eligible(const TailSeg &sg, int32_t max_rows) {
    return max_rows > 0 && sg.nrows > 0 && sg.nrows <= std::min(max_rows, kCodegenMaxRows) &&
           sg.nrows <= sg.W - sg.T;   // every in-segment term is a window slot
}

// The generator proper, on host copies of a segment's records.
sptrsv_status_t source_from_records(int32_t nr, int32_t K, int32_t nlev, const int32_t *row,
                                    const int32_t *nn, const int4 *term, const double2 *dg,
                                    std::string &src, bool &thin) {
    (void)K;
    int64_t terms = 0;
    for (int32_t p = 0; p < nr; ++p) {
        if ((nn[p] >> 8) & 0xFFFF) {   // a term read from x: not a window slot
            thin = false;
            return SPTRSV_OK;
        }
        terms += nn[p] & 0xFF;
    }
    // one thread pays every FMA in turn: worth it while a level averages
    // fewer than 16 terms (the record-driven kernel's barrier and row cost)
    thin = terms + nr < 16 * (int64_t)nlev;
    if (!thin) return SPTRSV_OK;
    src.clear();
    src.reserve((size_t)(terms * 48 + (int64_t)nr * 96 + 512));
    // one non-inlined function per kRowsPerFn rows: the compiler's time grows
    // much faster than linearly with the length of one straight-line body
    // (measured: 1,000 rows in one function 66 s, in functions of 50 rows
    // 1.3 s)
    char line[200];
    std::vector<std::pair<int32_t, double>> tk;
    const int32_t nfn = (nr + kRowsPerFn - 1) / kRowsPerFn;
    for (int32_t f = 0; f < nfn; ++f) {
        const int32_t p0 = f * kRowsPerFn, p1 = std::min(nr, p0 + kRowsPerFn);
        std::snprintf(line, sizeof line,
                      "__device__ __noinline__ void g%d(const double *__restrict__ s0, "
                      "double *__restrict__ x) {\n"
                      "  extern __shared__ double xs[];\n"
                      "  double v[%d];\n"
                      "  double a;\n",
                      f, kRowsPerFn);
        src += line;
        for (int32_t p = p0; p < p1; ++p) {
            const int cnt = nn[p] & 0xFF;
            tk.clear();
            for (int k = 0; k < cnt; ++k) {
                const int4 t = term[(size_t)k * nr + p];
                tk.emplace_back(t.x, from_halves(t.z, t.w));
            }
            // oldest unknowns first: the latest one closes the row's chain
            std::sort(tk.begin(), tk.end(),
                      [](const std::pair<int32_t, double> &u,
                         const std::pair<int32_t, double> &w) { return u.first < w.first; });
            std::snprintf(line, sizeof line, "  a = s0[%d];\n", p);
            src += line;
            for (const auto &t : tk) {
                const int32_t q = t.first;
                src += "  a = fma(";
                src += literal(-t.second);
                if (q >= p0)   // solved in this function: still in a register
                    std::snprintf(line, sizeof line, ", v[%d], a);\n", q - p0);
                else
                    std::snprintf(line, sizeof line, ", xs[%d], a);\n", q);
                src += line;
            }
            if (nn[p] & kTailUnscaled) {
                src += "  a = __ddiv_rn(a, ";
                src += literal(dg[p].x);
                src += ");\n";
            }
            std::snprintf(line, sizeof line, "  v[%d] = a; xs[%d] = a; x[%d] = a;\n", p - p0,
                          p, row[p]);
            src += line;
        }
        src += "}\n";
    }
    src += "extern \"C\" __global__ void __launch_bounds__(32) ";
    src += codegen_entry_name();
    src += "(const double *__restrict__ s0, double *__restrict__ x) {\n"
           "  if (threadIdx.x != 0) return;\n";
    for (int32_t f = 0; f < nfn; ++f) {
        std::snprintf(line, sizeof line, "  g%d(s0, x);\n", f);
        src += line;
    }
    src += "}\n";
    return SPTRSV_OK;
}


sptrsv_status_t codegen_source(const TailSeg &sg, std::string &src, bool &thin) {
    const int32_t nr = sg.nrows, K = sg.K;
    std::vector<int32_t> row(nr), nn(nr);
    std::vector<int4> term((size_t)K * nr);
    std::vector<double2> dg(nr);
    if (cudaMemcpy(row.data(), sg.row.p, sizeof(int32_t) * nr, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(nn.data(), sg.nn.p, sizeof(int32_t) * nr, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(term.data(), sg.term.p, sizeof(int4) * term.size(), cudaMemcpyDeviceToHost) !=
            cudaSuccess ||
        cudaMemcpy(dg.data(), sg.diag.p, sizeof(double2) * nr, cudaMemcpyDeviceToHost) !=
            cudaSuccess)
        return SPTRSV_ERR_CUDA;
    return source_from_records(nr, K, sg.nlev, row.data(), nn.data(), term.data(), dg.data(),
                               src, thin);
}

sptrsv_status_t codegen_build(TailSeg &sg, double &ms) {
    const auto t0 = std::chrono::steady_clock::now();
    sg.gen.reset();
    std::string src;
    bool thin = false;
    sptrsv_status_t st = codegen_source(sg, src, thin);
    if (st != SPTRSV_OK || !thin) return st;
    NvrtcApi &api = nvrtc();
    if (!api.ok) return SPTRSV_ERR_CODEGEN;
    nvrtcProgram prog;
    if (api.create(&prog, src.c_str(), "sptrsv_gen.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
        return SPTRSV_ERR_CODEGEN;
    const char *opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "--fmad=true"};
    const nvrtcResult cr = api.compile(prog, 3, opts);
    std::vector<char> cubin;
    if (cr == NVRTC_SUCCESS) {
        size_t n = 0;
        if (api.cubin_size(prog, &n) == NVRTC_SUCCESS && n > 0) {
            cubin.resize(n);
            if (api.cubin(prog, cubin.data()) != NVRTC_SUCCESS) cubin.clear();
        }
    }
    api.destroy(&prog);
    if (cubin.empty()) return SPTRSV_ERR_CODEGEN;
    GenKernel g;
    if (cudaLibraryLoadData(&g.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) !=
            cudaSuccess ||
        cudaLibraryGetKernel(&g.fn, g.lib, codegen_entry_name()) != cudaSuccess) {
        cudaGetLastError();
        return SPTRSV_ERR_CODEGEN;
    }
    g.smem = (size_t)sg.nrows * sizeof(double);
    if (g.smem > 48 * 1024 &&
        cudaFuncSetAttribute(reinterpret_cast<const void *>(g.fn),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem) !=
            cudaSuccess) {
        cudaGetLastError();
        return SPTRSV_ERR_CODEGEN;
    }
    sg.gen = std::move(g);
    ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return SPTRSV_OK;
}

cudaError_t codegen_launch(const TailSeg &sg, const double *b, double *x, cudaStream_t s) {
    cudaError_t e = launch_tail_fold(tail_view(sg), b, x, s);
    if (e != cudaSuccess) return e;
    const double *s0 = sg.s0.p;
    void *args[] = {(void *)&s0, (void *)&x};
    return cudaLaunchKernel(reinterpret_cast<const void *>(sg.gen.fn), dim3(1), dim3(32), args,
                            sg.gen.smem, s);
}

}  // namespace sptrsv

extern "C" SPTRSV_API sptrsv_status_t sptrsv_codegen_source_from_records(
    int32_t nrows, int32_t K, int32_t nlev, const int32_t *h_row, const int32_t *h_nn,
    const int32_t *h_term, const double *h_diag, char *buf, size_t cap, size_t *len) {
    if (nrows <= 0 || K <= 0 || K > 16 || nlev <= 0 || !h_row || !h_nn || !h_term || !h_diag ||
        !len)
        return SPTRSV_ERR_INVALID_ARG;
    for (int32_t p = 0; p < nrows; ++p) {   // every slot within the segment, counts <= K
        const int cnt = h_nn[p] & 0xFF;
        if (cnt > K) return SPTRSV_ERR_INVALID_ARG;
        for (int k = 0; k < cnt; ++k) {
            const int32_t q = h_term[4 * ((size_t)k * nrows + p)];
            if (!((h_nn[p] >> (8 + k)) & 1) && (q < 0 || q >= p)) return SPTRSV_ERR_INVALID_ARG;
        }
    }
    std::string src;
    bool thin = false;
    const sptrsv_status_t st = sptrsv::source_from_records(
        nrows, K, nlev, h_row, h_nn, reinterpret_cast<const int4 *>(h_term),
        reinterpret_cast<const double2 *>(h_diag), src, thin);
    if (st != SPTRSV_OK) return st;
    if (!thin) return SPTRSV_ERR_BAD_STATE;
    *len = src.size();
    if (buf && cap > 0) {
        const size_t k = std::min(cap - 1, src.size());
        std::memcpy(buf, src.data(), k);
        buf[k] = 0;
    }
    return SPTRSV_OK;
}
