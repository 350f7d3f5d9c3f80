// Batched solve of many plans in one persistent launch, captured in a CUDA
// graph on the first call (host side; the kernel is in solve.cu).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <queue>
#include <vector>

#include "plan.cuh"

using namespace sptrsv;

struct sptrsv_batch_s {
    std::vector<sptrsv_plan_t> plans;
    std::vector<double> lnorm;           // |L|_inf of every plan
    int device = 0;
    int num_sms = 0;
    bool ir = false;
    double tol = 1e-15;
    int max_iter = 8;
    uint64_t timeout_ns = 0;
    int block_threads = 256;
    int grid = 0;
    DevArr<BatchMat> d_mats;
    DevArr<BatchCtl> d_ctl;
    DevArr<DevStatus> st;
    BatchMat *h_mats = nullptr;          // pinned staging of the matrix table
    DevArr<float> d32;
    DevArr<double> r64;
    int64_t scratch_elems = 0;
    cudaGraphExec_t exec = nullptr;
    bool use_graph = true;
    bool graph_built = false;
    cudaStream_t graph_stream = nullptr;
    cudaEvent_t done = nullptr;
    bool launched = false;
    sptrsv_status_t latched = SPTRSV_OK;
    // CTA groups re-sized from the measured times of a first solve, valid for
    // the column counts they were measured with
    std::vector<int32_t> tuned_cnt, tuned_nrhs;
    ~sptrsv_batch_s() {
        if (exec) cudaGraphExecDestroy(exec);
        if (done) cudaEventDestroy(done);
        if (h_mats) cudaFreeHost(h_mats);
    }
};

namespace {

sptrsv_status_t cuda_err(cudaError_t e) {
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? SPTRSV_ERR_OOM : SPTRSV_ERR_CUDA;
}
#define BCK(x)                                                                 \
    do {                                                                       \
        cudaError_t _e = (x);                                                  \
        if (_e != cudaSuccess) return cuda_err(_e);                            \
    } while (0)

int pow2_at_least(int v) {
    int r = 1;
    while (r < v) r <<= 1;
    return r;
}

// Predicted time of one matrix's solve on w warps, in chunk passes: the
// levels run one after another and a level of C chunks takes ceil(C / w)
// passes of the group's warps (its critical path times its width), plus the
// work that is not tied to levels (refinement sweeps, the copy of x), spread
// over all w warps; `work` is counted in chunk passes of one warp.
double predict_passes(const std::vector<int32_t> &lvl_chunk, double work, int64_t w) {
    double t = 0.0;
    for (size_t l = 0; l + 1 < lvl_chunk.size(); ++l) {
        const int64_t c = lvl_chunk[l + 1] - lvl_chunk[l];
        t += (double)((c + w - 1) / w);
    }
    return t + work / (double)w;
}

// Splits `total` CTAs (warps_per_cta warps each) over the matrices, at least
// one each, so that the slowest predicted matrix is as fast as it can be:
// the matrix predicted slowest gets the next CTA while that shortens its
// time.  CTAs that shorten no matrix go in proportion to `bytes`.
// `scale` (optional) turns each prediction into time: a matrix measured at
// t ms on c CTAs gets scale t / predict(c).
bool assign_groups_by_time(const std::vector<const std::vector<int32_t> *> &lvl,
                           const std::vector<double> &work, const std::vector<double> &bytes,
                           int total, int warps_per_cta, std::vector<int32_t> &cnt,
                           const std::vector<double> *scale = nullptr) {
    const int m = (int)lvl.size();
    if (m > total) return false;
    cnt.assign(m, 1);
    std::vector<double> t(m);
    auto sc = [&](int i) { return scale ? (*scale)[i] : 1.0; };
    std::priority_queue<std::pair<double, int>> heap;
    for (int i = 0; i < m; ++i) {
        t[i] = sc(i) * predict_passes(*lvl[i], work[i], warps_per_cta);
        heap.emplace(t[i], i);
    }
    int left = total - m;
    while (left > 0 && !heap.empty()) {
        const int i = heap.top().second;
        heap.pop();
        const double tn =
            sc(i) * predict_passes(*lvl[i], work[i], (int64_t)(cnt[i] + 1) * warps_per_cta);
        if (tn >= t[i] - 1e-9) continue;   // saturated: one pass per level already
        cnt[i] += 1;
        t[i] = tn;
        --left;
        heap.emplace(t[i], i);
    }
    if (left > 0) {   // the rest by bytes
        double sum = 0.0;
        for (double v : bytes) sum += v;
        for (int i = 0; i < m && sum > 0.0; ++i) cnt[i] += (int)std::floor(bytes[i] / sum * left);
    }
    return true;
}


}  // namespace

extern "C" {

SPTRSV_API sptrsv_status_t sptrsv_batch_create(const sptrsv_plan_t *plans, int32_t count,
                                               sptrsv_batch_t *out) {
    if (!out || count < 1 || !plans) return SPTRSV_ERR_INVALID_ARG;
    *out = nullptr;
    int dev = 0;
    BCK(cudaGetDevice(&dev));
    const bool ir = plans[0] && plans[0]->prm.precision == SPTRSV_F32_IR;
    for (int32_t i = 0; i < count; ++i) {
        const sptrsv_plan_t p = plans[i];
        if (!p) return SPTRSV_ERR_INVALID_ARG;
        if (p->latched != SPTRSV_OK) return SPTRSV_ERR_BAD_STATE;
        if (p->device != dev) return SPTRSV_ERR_INVALID_ARG;
        if ((p->prm.precision == SPTRSV_F32_IR) != ir) return SPTRSV_ERR_INVALID_ARG;
        if (p->n > 0 && (ir ? !p->s32.built : !p->s64.built)) return SPTRSV_ERR_BAD_STATE;
    }
    sptrsv_batch_s *bt = new sptrsv_batch_s();
    bt->plans.assign(plans, plans + count);
    bt->lnorm.resize(count);
    for (int32_t i = 0; i < count; ++i) {
        unsigned long long lb = 0;
        cudaError_t e = cudaMemcpy(&lb, plans[i]->lnorm.p, sizeof(lb), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            delete bt;
            return cuda_err(e);
        }
        std::memcpy(&bt->lnorm[i], &lb, sizeof(double));
    }
    bt->device = dev;
    bt->ir = ir;
    BCK(cudaDeviceGetAttribute(&bt->num_sms, cudaDevAttrMultiProcessorCount, dev));
    const sptrsv_plan_t p0 = plans[0];
    bt->tol = p0->prm.ir_tol;
    bt->max_iter = std::min(p0->prm.ir_max_iter, kBatchMaxIter);
    bt->timeout_ns = (uint64_t)(p0->prm.wait_timeout_ms > 0 ? p0->prm.wait_timeout_ms : 5000) *
                     1000000ull;
    bt->block_threads = 256;
    const int mx = batch_max_coresident(ir, bt->block_threads, bt->num_sms);
    if (mx < count) {
        delete bt;
        return mx <= 0 ? SPTRSV_ERR_CUDA : SPTRSV_ERR_UNSUPPORTED;
    }
    bt->grid = mx;
    auto fail = [&](cudaError_t e) {
        delete bt;
        return cuda_err(e);
    };
    cudaError_t e;
    if ((e = bt->d_mats.alloc(count)) != cudaSuccess) return fail(e);
    if ((e = bt->d_ctl.alloc(count)) != cudaSuccess) return fail(e);
    if ((e = bt->st.alloc(1)) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(bt->st.p, 0, sizeof(DevStatus))) != cudaSuccess) return fail(e);
    if ((e = cudaMallocHost((void **)&bt->h_mats, sizeof(BatchMat) * count)) != cudaSuccess)
        return fail(e);
    if ((e = cudaEventCreateWithFlags(&bt->done, cudaEventDisableTiming)) != cudaSuccess)
        return fail(e);
    *out = bt;
    return SPTRSV_OK;
}

SPTRSV_API sptrsv_status_t sptrsv_batch_solve(sptrsv_batch_t bt, const double *const *d_b,
                                              double *const *d_x, const int32_t *nrhs,
                                              sptrsv_stream_t stream) {
    if (!bt || !d_b || !d_x || !nrhs) return SPTRSV_ERR_INVALID_ARG;
    if (bt->latched != SPTRSV_OK) return SPTRSV_ERR_BAD_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t m = (int32_t)bt->plans.size();
    // scratch for the refinement: one [n, nrhs] FP32 + FP64 pair per matrix
    std::vector<int64_t> off(m + 1, 0);
    std::vector<double> w(m);
    for (int32_t i = 0; i < m; ++i) {
        const sptrsv_plan_t p = bt->plans[i];
        if (nrhs[i] < 1 || nrhs[i] > 32) return SPTRSV_ERR_INVALID_ARG;
        if (p->n > 0 && (!d_b[i] || !d_x[i])) return SPTRSV_ERR_INVALID_ARG;
        off[i + 1] = off[i] + (int64_t)p->n * nrhs[i];
        const int64_t slots = bt->ir ? p->s32.nslots : p->s64.nslots;
        w[i] = (double)slots * (bt->ir ? 8 : 12) + (double)p->n * (16.0 + 16.0 * nrhs[i]);
    }
    // groups sized by predicted time: levels (critical path) x chunks per level
    std::vector<const std::vector<int32_t> *> lvl(m);
    std::vector<double> work(m);
    for (int32_t i = 0; i < m; ++i) {
        const sptrsv_plan_t p = bt->plans[i];
        lvl[i] = bt->ir ? &p->s32.h_lvl_chunk : &p->s64.h_lvl_chunk;
        // refinement sweeps and copies: about a chunk pass per 32 x 8 row-columns per round
        const int rounds = bt->ir ? 3 : 1;
        work[i] = (double)p->n * nrhs[i] * rounds / 256.0;
    }
    std::vector<int32_t> cnt;
    const std::vector<int32_t> nr_now(nrhs, nrhs + m);
    const bool tuned = !bt->tuned_cnt.empty() && bt->tuned_nrhs == nr_now;
    if (tuned) cnt = bt->tuned_cnt;
    else if (!assign_groups_by_time(lvl, work, w, bt->grid, bt->block_threads / 32, cnt))
        return SPTRSV_ERR_UNSUPPORTED;
    // the staging table may still be read by the previous launch
    if (bt->launched) BCK(cudaEventSynchronize(bt->done));
    if (bt->ir && off[m] > bt->scratch_elems) {
        BCK(bt->d32.alloc(off[m]));
        BCK(bt->r64.alloc(off[m]));
        bt->scratch_elems = off[m];
        bt->graph_built = false;  // the captured graph points at the old scratch
    }
    auto fill_table = [&](const std::vector<int32_t> &cnt) {
    int32_t begin = 0;
    for (int32_t i = 0; i < m; ++i) {
        const sptrsv_plan_t p = bt->plans[i];
        BatchMat &M = bt->h_mats[i];
        std::memset(&M, 0, sizeof(M));
        if (bt->ir) {
            M.s32 = p->s32.view();
        } else {
            M.s64 = p->s64.view();
        }
        M.row_ptr = p->row_ptr.p;
        M.col = p->col.p;
        M.val = p->val.p;
        M.rev = p->rev ? 1 : 0;
        M.b = d_b[i];
        M.x = d_x[i];
        M.d32 = bt->ir ? bt->d32.p + off[i] : nullptr;
        M.r64 = bt->ir ? bt->r64.p + off[i] : nullptr;
        M.lnorm = bt->lnorm[i];
        M.n = p->n;
        M.nr = nrhs[i];
        M.R = pow2_at_least(nrhs[i]);
        M.cta_begin = begin;
        M.cta_count = cnt[i];
        begin += cnt[i];
    }
    };
    fill_table(cnt);
    auto enqueue = [&](cudaStream_t q) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(bt->d_mats.p, bt->h_mats, sizeof(BatchMat) * m,
                                        cudaMemcpyHostToDevice, q);
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(bt->d_ctl.p, 0, sizeof(BatchCtl) * m, q);
        if (e != cudaSuccess) return e;
        return launch_batch(bt->d_mats.p, m, bt->d_ctl.p, bt->st.p, bt->ir, bt->tol, bt->max_iter,
                            bt->timeout_ns, bt->block_threads, bt->grid, q);
    };
    if (!tuned) {
        // first solve with these column counts: run it once, measure every
        // group, and re-size the groups from the measured times
        BCK(enqueue(s));
        BCK(cudaStreamSynchronize(s));
        std::vector<BatchCtl> ctl(m);
        BCK(cudaMemcpy(ctl.data(), bt->d_ctl.p, sizeof(BatchCtl) * m, cudaMemcpyDeviceToHost));
        std::vector<double> scale(m, 1.0);
        const int wpc = bt->block_threads / 32;
        for (int32_t i = 0; i < m; ++i) {
            const double ms = ctl[i].t_end > ctl[i].t_begin
                                  ? (double)(ctl[i].t_end - ctl[i].t_begin) * 1e-6 : 0.0;
            const double pr = predict_passes(*lvl[i], work[i], (int64_t)cnt[i] * wpc);
            scale[i] = pr > 0.0 ? ms / pr : 0.0;
        }
        std::vector<int32_t> cnt2;
        if (assign_groups_by_time(lvl, work, w, bt->grid, wpc, cnt2, &scale)) {
            cnt = cnt2;
            fill_table(cnt);
        }
        bt->tuned_cnt = cnt;
        bt->tuned_nrhs = nr_now;
        bt->graph_built = false;   // capture the re-sized table
    }
    // the legacy default stream cannot be captured: launch directly there
    if (bt->use_graph && s != nullptr && (!bt->graph_built || bt->graph_stream != s)) {
        if (bt->exec) {
            cudaGraphExecDestroy(bt->exec);
            bt->exec = nullptr;
        }
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = enqueue(s);
            e = cudaStreamEndCapture(s, &g);
            if (e2 != cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&bt->exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            bt->use_graph = false;  // capture unsupported here: launch directly
            if (bt->exec) cudaGraphExecDestroy(bt->exec);
            bt->exec = nullptr;
        } else {
            bt->graph_built = true;
            bt->graph_stream = s;
        }
    }
    if (bt->use_graph && bt->graph_built && s == bt->graph_stream) {
        BCK(cudaGraphLaunch(bt->exec, s));
    } else {
        BCK(enqueue(s));
    }
    BCK(cudaEventRecord(bt->done, s));
    bt->launched = true;
    return SPTRSV_OK;
}

SPTRSV_API sptrsv_status_t sptrsv_batch_check(sptrsv_batch_t bt, sptrsv_stream_t stream) {
    if (!bt) return SPTRSV_ERR_INVALID_ARG;
    if (bt->latched != SPTRSV_OK) return bt->latched;
    BCK(cudaStreamSynchronize((cudaStream_t)stream));
    DevStatus h;
    BCK(cudaMemcpy(&h, bt->st.p, sizeof(h), cudaMemcpyDeviceToHost));
    if (h.code) bt->latched = (sptrsv_status_t)h.code;
    return bt->latched;
}

SPTRSV_API sptrsv_status_t sptrsv_batch_get_info(sptrsv_batch_t bt, int32_t *h_iters,
                                                 int32_t *h_converged, int32_t *h_cta_count,
                                                 int32_t *h_graph) {
    if (!bt) return SPTRSV_ERR_INVALID_ARG;
    const int32_t m = (int32_t)bt->plans.size();
    if (bt->launched) BCK(cudaEventSynchronize(bt->done));
    std::vector<BatchCtl> ctl(m);
    BCK(cudaMemcpy(ctl.data(), bt->d_ctl.p, sizeof(BatchCtl) * m, cudaMemcpyDeviceToHost));
    for (int32_t i = 0; i < m; ++i) {
        if (h_iters) h_iters[i] = ctl[i].iters;
        if (h_converged) h_converged[i] = ctl[i].converged;
        if (h_cta_count) h_cta_count[i] = bt->h_mats[i].cta_count;
    }
    if (h_graph) *h_graph = (bt->use_graph && bt->graph_built) ? 1 : 0;
    return SPTRSV_OK;
}

SPTRSV_API sptrsv_status_t sptrsv_batch_get_times(sptrsv_batch_t bt, float *h_ms) {
    if (!bt || !h_ms) return SPTRSV_ERR_INVALID_ARG;
    const int32_t m = (int32_t)bt->plans.size();
    if (!bt->launched) return SPTRSV_ERR_BAD_STATE;
    BCK(cudaEventSynchronize(bt->done));
    std::vector<BatchCtl> ctl(m);
    BCK(cudaMemcpy(ctl.data(), bt->d_ctl.p, sizeof(BatchCtl) * m, cudaMemcpyDeviceToHost));
    for (int32_t i = 0; i < m; ++i)
        h_ms[i] = ctl[i].t_end > ctl[i].t_begin
                      ? (float)((double)(ctl[i].t_end - ctl[i].t_begin) * 1e-6) : 0.f;
    return SPTRSV_OK;
}

SPTRSV_API void sptrsv_batch_destroy(sptrsv_batch_t bt) {
    if (!bt) return;
    if (bt->launched) cudaEventSynchronize(bt->done);
    delete bt;
}

}  // extern "C"
