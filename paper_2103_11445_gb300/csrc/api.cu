// C entry points: plan life cycle, analysis and transform orchestration,
// the thin-level selection heuristic, the solve dispatcher and the
// launch-configuration autotuner.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include "codegen.cuh"
#include "plan.cuh"
#include "tail.cuh"

using namespace sptrsv;

namespace sptrsv {
// mlp.cu: normalise h_feat [count][16] and run the network, h_pred[count]
sptrsv_mlp_t default_costmodel();   // mlp.cu: the process-wide network, or null
sptrsv_mlp_t default_segmodel();    // mlp.cu: the per-segment network, or null
sptrsv_status_t costmodel_predict(sptrsv_mlp_t net, const float *h_feat, int count,
                                  float *h_pred, cudaStream_t s);
}

namespace {

sptrsv_status_t cuda_status(cudaError_t e) {
    return e == cudaErrorMemoryAllocation ? SPTRSV_ERR_OOM : SPTRSV_ERR_CUDA;
}

#define CK(x)                                                                  \
    do {                                                                       \
        cudaError_t _e = (x);                                                  \
        if (_e != cudaSuccess) {                                               \
            (void)cudaGetLastError();                                          \
            return cuda_status(_e);                                            \
        }                                                                      \
    } while (0)
#define CKS(x)                                                                 \
    do {                                                                       \
        sptrsv_status_t _s = (x);                                              \
        if (_s != SPTRSV_OK) return _s;                                        \
    } while (0)

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

uint64_t timeout_ns(const sptrsv_plan_s *p) {
    const int ms = p->prm.wait_timeout_ms > 0 ? p->prm.wait_timeout_ms : 5000;
    return (uint64_t)ms * 1000000ull;
}

template <typename T>
cudaError_t upload(DevArr<T> &d, const std::vector<T> &h, cudaStream_t s) {
    cudaError_t e = d.alloc(h.size());
    if (e != cudaSuccess || h.empty()) return e;
    return cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

// Synchronise and surface a device-latched error.
sptrsv_status_t sync_status(sptrsv_plan_t p, cudaStream_t s) {
    CK(cudaStreamSynchronize(s));
    DevStatus h;
    CK(cudaMemcpy(&h, p->status.p, sizeof(h), cudaMemcpyDeviceToHost));
    if (h.code != 0) {
        p->latched = (sptrsv_status_t)h.code;
        return p->latched;
    }
    return SPTRSV_OK;
}

// ---------------------------------------------------------------------------
// Thin-level selection heuristic H (the row choice the paper leaves to the
// programmer, Sec. IV; its experiment removes thin levels at +10% FLOPs,
// Sec. V).  Levels are scanned in order; a segment starts at a kept level t
// and absorbs t+1, t+2, ... while the next level is thin (< tau rows), fewer
// than d_max levels were absorbed, the rewrite fits the fill cap and the
// FLOPs added over the whole matrix stay within rho * base_flops.
// added(l, r, &cost) returns false when a row of level l would exceed the
// fill cap when lifted to level l - r.
std::vector<std::pair<int32_t, int32_t>> select_segments(
    const std::vector<int64_t> &level_rows, int64_t tau, int32_t d_max, double rho,
    int64_t base_flops, const std::function<bool(int32_t, int32_t, int64_t *)> &added) {
    const int32_t nlev = (int32_t)level_rows.size();
    const double budget = rho * (double)base_flops;
    int64_t used = 0;
    std::vector<std::pair<int32_t, int32_t>> segs;
    int32_t lv = 0;
    while (lv < nlev) {
        const int32_t t = lv;
        int32_t d = 0;
        while (d < d_max && t + d + 1 < nlev && level_rows[t + d + 1] < tau) {
            int64_t cost = 0;
            if (!added(t + d + 1, d + 1, &cost)) break;
            if ((double)(used + cost) > budget) break;
            used += cost;
            ++d;
        }
        segs.emplace_back(t, d);
        lv = t + d + 1;
    }
    return segs;
}

// Evaluates candidate rewrites (level l lifted by r levels) on the device,
// in batches, caching the results.
struct FillQuery {
    sptrsv_plan_t p;
    cudaStream_t s;
    int cap;
    std::map<std::pair<int32_t, int32_t>, int64_t> cache;  // -1: overflow
    std::map<std::pair<int32_t, int32_t>, int32_t> maxlen;  // most terms of a lifted row
    sptrsv_status_t err = SPTRSV_OK;

    sptrsv_status_t run(const std::vector<std::pair<int32_t, int32_t>> &qs_in) {
        std::vector<int32_t> ql, qt;
        std::vector<int64_t> qoff(1, 0);
        for (auto &q : qs_in) {
            if (cache.count(q)) continue;
            const int32_t l = q.first, r = q.second;
            ql.push_back(l);
            qt.push_back(l - r);
            qoff.push_back(qoff.back() + (p->h_level_ptr[l + 1] - p->h_level_ptr[l]));
            cache[q] = -2;  // placeholder, filled below
        }
        const int32_t nq = (int32_t)ql.size();
        if (nq == 0) return SPTRSV_OK;
        const int64_t nitems = qoff.back();
        DevArr<int32_t> d_ql, d_qt, irow, itgt, iq, ovf, mlen;
        DevArr<int64_t> d_qoff;
        DevArr<unsigned long long> added;
        CK(upload(d_ql, ql, s));
        CK(upload(d_qt, qt, s));
        CK(upload(d_qoff, qoff, s));
        CK(irow.alloc(nitems));
        CK(itgt.alloc(nitems));
        CK(iq.alloc(nitems));
        CK(ovf.alloc(nq));
        CK(mlen.alloc(nq));
        CK(added.alloc(nq));
        CK(cudaMemsetAsync(ovf.p, 0, nq * sizeof(int32_t), s));
        CK(cudaMemsetAsync(mlen.p, 0, nq * sizeof(int32_t), s));
        CK(cudaMemsetAsync(added.p, 0, nq * sizeof(unsigned long long), s));
        CK(launch_expand_queries(nq, d_ql.p, d_qt.p, d_qoff.p, p->level_ptr.p, p->perm.p, irow.p,
                                 itgt.p, iq.p, nullptr, s));
        CK(launch_rewrite_count(nitems, irow.p, itgt.p, iq.p, p->row_ptr.p, p->col.p,
                                p->level.p, cap, nullptr, added.p, ovf.p, mlen.p, p->num_sms,
                                s));
        std::vector<int32_t> h_ovf(nq), h_mlen(nq);
        std::vector<unsigned long long> h_add(nq);
        CK(cudaMemcpyAsync(h_ovf.data(), ovf.p, nq * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(h_add.data(), added.p, nq * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(h_mlen.data(), mlen.p, nq * sizeof(int32_t), cudaMemcpyDeviceToHost,
                           s));
        CK(cudaStreamSynchronize(s));
        for (int32_t i = 0; i < nq; ++i) {
            cache[{ql[i], ql[i] - qt[i]}] = h_ovf[i] ? -1 : (int64_t)h_add[i];
            maxlen[{ql[i], ql[i] - qt[i]}] = h_mlen[i];
        }
        return SPTRSV_OK;
    }

    // the rewrites H would query if nothing were cut, from segment start t
    void optimistic_from(int32_t t, const std::vector<int64_t> &rows, int64_t tau, int32_t d_max,
                         std::vector<std::pair<int32_t, int32_t>> &out) const {
        const int32_t nlev = (int32_t)rows.size();
        while (t < nlev) {
            int32_t d = 0;
            while (d < d_max && t + d + 1 < nlev && rows[t + d + 1] < tau) {
                out.emplace_back(t + d + 1, d + 1);
                ++d;
            }
            t += d + 1;
        }
    }
};

int64_t plain_flops(const sptrsv_plan_s *p) { return 2 * (p->nnz - p->n) + p->n; }

// Segments chosen by H for (tau, d_max, rho), with the FLOPs they add;
// leaves the plan untouched.
sptrsv_status_t compute_segments(sptrsv_plan_t p, int64_t tau, int32_t d_max, double rho,
                                 cudaStream_t s, std::vector<std::pair<int32_t, int32_t>> *out,
                                 int64_t *added_flops) {
    const int32_t nlev = p->nlev;
    std::vector<int64_t> rows(nlev);
    for (int32_t l = 0; l < nlev; ++l) rows[l] = p->h_level_ptr[l + 1] - p->h_level_ptr[l];
    FillQuery fo{p, s, p->prm.max_row_fill, {}};
    // speculative batch: the uncut path plus every first step after a cut
    std::vector<std::pair<int32_t, int32_t>> qs;
    fo.optimistic_from(0, rows, tau, d_max, qs);
    if (d_max > 0 && std::isfinite(rho))
        for (int32_t l = 1; l < nlev; ++l)
            if (rows[l] < tau) qs.emplace_back(l, 1);
    CKS(fo.run(qs));
    auto added = [&](int32_t l, int32_t r, int64_t *cost) -> bool {
        auto it = fo.cache.find({l, r});
        if (it == fo.cache.end()) {
            std::vector<std::pair<int32_t, int32_t>> more;
            fo.optimistic_from(l - r, rows, tau, d_max, more);
            more.emplace_back(l, r);
            fo.err = fo.run(more);
            it = fo.cache.find({l, r});
            if (fo.err != SPTRSV_OK || it == fo.cache.end()) return false;
        }
        if (it->second < 0) return false;
        *cost = it->second;
        return true;
    };
    *out = select_segments(rows, tau, d_max, rho, plain_flops(p), added);
    if (fo.err != SPTRSV_OK) return fo.err;
    int64_t tot = 0;
    for (auto &sg : *out)
        for (int32_t r = 1; r <= sg.second; ++r) tot += fo.cache[{sg.first + r, r}];
    *added_flops = tot;
    return SPTRSV_OK;
}

// SELECT_CRITPATH: the segmentation minimising the level-set critical path
// sum over new levels of (hop + most terms of a row in it), by dynamic
// programming over the levels, last first, ties to the smaller depth; every
// lift (l, r <= d_max) is counted on the device first.
sptrsv_status_t critpath_segments(sptrsv_plan_t p, int64_t hop, int32_t d_max, cudaStream_t s,
                                  std::vector<std::pair<int32_t, int32_t>> *out) {
    const int32_t nlev = p->nlev;
    std::vector<int32_t> lm0(nlev, 0);
    {
        DevArr<int32_t> lm;
        CK(lm.alloc(nlev));
        CK(cudaMemsetAsync(lm.p, 0, nlev * sizeof(int32_t), s));
        CK(launch_level_max(p->n, p->level.p, p->offdeg.p, lm.p, s));
        CK(cudaMemcpyAsync(lm0.data(), lm.p, nlev * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    FillQuery fo{p, s, p->prm.max_row_fill, {}};
    std::vector<std::pair<int32_t, int32_t>> qs;
    for (int32_t l = 1; l < nlev; ++l)
        for (int32_t r = 1; r <= std::min(d_max, l); ++r) qs.emplace_back(l, r);
    CKS(fo.run(qs));
    std::vector<double> best(nlev + 1, INFINITY);
    std::vector<int32_t> choice(nlev + 1, 0);
    best[nlev] = 0.0;
    for (int32_t t = nlev - 1; t >= 0; --t) {
        int64_t m = lm0[t];
        for (int32_t d = 0; d <= d_max && t + d < nlev; ++d) {
            if (d > 0) {
                if (fo.cache[{t + d, d}] < 0) break;   // a row would exceed the fill cap
                m = std::max<int64_t>(m, fo.maxlen[{t + d, d}]);
            }
            const double c = (double)(hop + m) + best[t + d + 1];
            if (c < best[t]) {
                best[t] = c;
                choice[t] = d;
            }
        }
    }
    out->clear();
    for (int32_t t = 0; t < nlev; t += choice[t] + 1) out->emplace_back(t, choice[t]);
    return SPTRSV_OK;
}

// Features of every candidate segment (t, d <= d_max) -- the analysis of
// the levels it merges and the lift counts of its rewritten rows (the
// matrix-analysis module's per-level view, Sec. IV), as the per-segment cost
// network of SELECT_SEGMODEL reads them:
//   0 log2(1 + rows), 1 log2(1 + x and b terms), 2 log2(1 + most terms of a
//   row), 3 terms per row, 4 d, 5 fraction of rows rewritten, 6 log2 n,
//   7 log2(nnz / n).
// ok[t * (d_max + 1) + d] = 0 where t + d runs past the last level or a
// lifted row would exceed the fill cap.
sptrsv_status_t segment_table(sptrsv_plan_t p, int32_t d_max, cudaStream_t s,
                              std::vector<float> &feat, std::vector<uint8_t> &ok) {
    const int32_t nlev = p->nlev, D = d_max + 1;
    feat.assign((size_t)nlev * D * kSegFeatures, 0.0f);
    ok.assign((size_t)nlev * D, 0);
    if (nlev == 0) return SPTRSV_OK;
    std::vector<int32_t> lm0(nlev, 0);
    std::vector<unsigned long long> acc((size_t)nlev * 11, 0);
    {
        DevArr<int32_t> lm;
        DevArr<unsigned long long> dacc;
        CK(lm.alloc(nlev));
        CK(dacc.alloc((size_t)nlev * 11));
        CK(cudaMemsetAsync(lm.p, 0, nlev * sizeof(int32_t), s));
        CK(cudaMemsetAsync(dacc.p, 0, (size_t)nlev * 11 * sizeof(unsigned long long), s));
        CK(launch_level_max(p->n, p->level.p, p->offdeg.p, lm.p, s));
        CK(launch_level_counts(p->n, p->row_ptr.p, p->col.p, p->level.p, dacc.p, s));
        CK(cudaMemcpyAsync(lm0.data(), lm.p, nlev * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(acc.data(), dacc.p, acc.size() * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    FillQuery fo{p, s, p->prm.max_row_fill, {}};
    std::vector<std::pair<int32_t, int32_t>> qs;
    for (int32_t l = 1; l < nlev; ++l)
        for (int32_t r = 1; r <= std::min(d_max, l); ++r) qs.emplace_back(l, r);
    CKS(fo.run(qs));
    const float ln = std::log2((float)std::max<int32_t>(p->n, 1));
    const float ld = std::log2((float)std::max<int64_t>(p->nnz, 1) / std::max<int32_t>(p->n, 1));
    for (int32_t t = 0; t < nlev; ++t) {
        double rows = 0, terms = 0, maxt = 0, rew = 0;
        for (int32_t d = 0; d <= d_max && t + d < nlev; ++d) {
            const int32_t l = t + d;
            const double rl = (double)acc[(size_t)l * 11 + 0];
            if (d == 0) {
                terms += (double)acc[(size_t)l * 11 + 1];
                maxt = lm0[t];
            } else {
                const int64_t add = fo.cache[{l, d}];
                if (add < 0) break;   // deeper merges lift this level too
                terms += (double)acc[(size_t)l * 11 + 1] + 0.5 * (double)add;
                maxt = std::max<double>(maxt, fo.maxlen[{l, d}]);
                rew += rl;
            }
            rows += rl;
            float *f = &feat[((size_t)t * D + d) * kSegFeatures];
            f[0] = (float)std::log2(1.0 + rows);
            f[1] = (float)std::log2(1.0 + terms);
            f[2] = (float)std::log2(1.0 + maxt);
            f[3] = (float)(terms / std::max(rows, 1.0));
            f[4] = (float)d;
            f[5] = (float)(rew / std::max(rows, 1.0));
            f[6] = ln;
            f[7] = ld;
            ok[(size_t)t * D + d] = 1;
        }
    }
    return SPTRSV_OK;
}

constexpr int32_t kSegMaxDepth = 4;   // deepest segment of the segment network's data

// SELECT_SEGMODEL: the network predicts the log2 time (us) each candidate
// segment adds to the solve; the segmentation minimising the sum, by
// dynamic programming over the levels as in SELECT_CRITPATH (ties to the
// smaller depth).
sptrsv_status_t segmodel_segments(sptrsv_plan_t p, sptrsv_mlp_t net, int32_t d_max,
                                  cudaStream_t s, std::vector<std::pair<int32_t, int32_t>> *out) {
    const int32_t nlev = p->nlev, D = d_max + 1;
    std::vector<float> feat;
    std::vector<uint8_t> ok;
    CKS(segment_table(p, d_max, s, feat, ok));
    std::vector<float> pred((size_t)nlev * D, 0.0f);
    // the feasible rows only, in one batch
    std::vector<float> fx;
    std::vector<int64_t> at;
    for (size_t i = 0; i < ok.size(); ++i)
        if (ok[i]) {
            fx.insert(fx.end(), feat.begin() + i * kSegFeatures,
                      feat.begin() + (i + 1) * kSegFeatures);
            at.push_back((int64_t)i);
        }
    std::vector<float> px(at.size());
    if (!at.empty()) CKS(costmodel_predict(net, fx.data(), (int)at.size(), px.data(), s));
    for (size_t k = 0; k < at.size(); ++k) pred[at[k]] = px[k];
    std::vector<double> best(nlev + 1, INFINITY);
    std::vector<int32_t> choice(nlev + 1, 0);
    best[nlev] = 0.0;
    for (int32_t t = nlev - 1; t >= 0; --t)
        for (int32_t d = 0; d <= d_max && t + d < nlev; ++d) {
            if (!ok[(size_t)t * D + d]) break;
            const double c = std::exp2((double)pred[(size_t)t * D + d]) + best[t + d + 1];
            if (c < best[t]) {
                best[t] = c;
                choice[t] = d;
            }
        }
    out->clear();
    for (int32_t t = 0; t < nlev; t += choice[t] + 1) out->emplace_back(t, choice[t]);
    return SPTRSV_OK;
}

// Candidate rewrite depths the cost model chooses from (0 = plain levels).
// Candidates of SELECT_COSTMODEL.  A code c < kThinOnly merges every c+1
// levels (c = 0: the plain level sets); c = kThinOnly + d rewrites only the
// levels of fewer than kThinRows rows (one warp), up to d of them into the
// level before, within kThinBudget times the plain FLOPs.
constexpr int kThinOnly = 100;
constexpr int kThinRows = 32;
constexpr double kThinBudget = 4.0;
constexpr int kCostDepths[] = {0, 1, 2, 3, 4, 6, 8, kThinOnly + 8, kThinOnly + 16};
constexpr int kNumCostDepths = 9;
constexpr int kCostFeatures = 17;

// Features of "merge every d+1 levels" on this plan (the analysis features
// of the matrix-analysis module, Sec. IV, plus the candidate's fill):
//  0 log2 n, 1 log2 nnz, 2 dependencies per row, 3 log2 levels,
//  4 log2 rows per level, 5-6 fraction of levels with < 32 / < 1024 rows,
//  7 fraction of rows in levels of < 1024 rows, 8-11 fraction of rows with
//  0 | 1-2 | 3-6 | >= 7 dependencies, 12 d, 13 log2 levels after,
//  14 FLOPs after / FLOPs before, 15 fraction of rows rewritten.
sptrsv_status_t candidate_features(sptrsv_plan_t p, int code, float *f, cudaStream_t s) {
    const bool thin_only = code >= kThinOnly;
    const int d = thin_only ? code - kThinOnly : code;
    const double n = std::max<int32_t>(p->n, 1), nnz = std::max<int64_t>(p->nnz, 1);
    const int32_t nlev = std::max<int32_t>(p->nlev, 1);
    int64_t thin32 = 0, thin1k = 0, rows1k = 0;
    for (int32_t l = 0; l < p->nlev; ++l) {
        const int64_t r = p->h_level_ptr[l + 1] - p->h_level_ptr[l];
        thin32 += r < 32;
        thin1k += r < 1024;
        rows1k += r < 1024 ? r : 0;
    }
    std::vector<std::pair<int32_t, int32_t>> segs;
    int64_t added = 0;
    if (d > 0 && p->nlev > 0) {
        if (thin_only) CKS(compute_segments(p, kThinRows, d, kThinBudget, s, &segs, &added));
        else CKS(compute_segments(p, INT64_MAX, d, INFINITY, s, &segs, &added));
    } else {
        for (int32_t l = 0; l < p->nlev; ++l) segs.emplace_back(l, 0);
    }
    int64_t rewritten = 0;
    for (auto &sg : segs)
        rewritten += p->h_level_ptr[sg.first + sg.second + 1] - p->h_level_ptr[sg.first + 1];
    const double fp = (double)std::max<int64_t>(plain_flops(p), 1);
    f[0] = (float)std::log2(n);
    f[1] = (float)std::log2(nnz);
    f[2] = (float)((p->nnz - p->n) / n);
    f[3] = (float)std::log2((double)nlev);
    f[4] = (float)std::log2(n / nlev);
    f[5] = (float)thin32 / nlev;
    f[6] = (float)thin1k / nlev;
    f[7] = (float)(rows1k / n);
    for (int k = 0; k < 4; ++k) f[8 + k] = (float)(p->offdeg_hist[k] / n);
    f[12] = (float)d;
    f[13] = (float)std::log2((double)std::max<size_t>(segs.size(), 1));
    f[14] = (float)((fp + added) / fp);
    f[15] = (float)(rewritten / n);
    f[16] = thin_only ? 1.0f : 0.0f;
    return SPTRSV_OK;
}

sptrsv_status_t choose_segments(sptrsv_plan_t p, cudaStream_t s) {
    const auto &prm = p->prm;
    const int32_t nlev = p->nlev;
    p->seg_first.clear();
    p->seg_depth.clear();
    p->chosen_depth = -1;
    if (prm.select_mode == SPTRSV_SELECT_NONE || nlev == 0) {
        for (int32_t l = 0; l < nlev; ++l) {
            p->seg_first.push_back(l);
            p->seg_depth.push_back(0);
        }
        return SPTRSV_OK;
    }
    int64_t tau;
    int32_t d_max;
    double rho;
    // the plan's network, else the process-wide one (sptrsv_costmodel_load)
    sptrsv_mlp_t net = p->costmodel ? p->costmodel : default_costmodel();
    if (prm.select_mode == SPTRSV_SELECT_COSTMODEL && net) {
        // the network predicts the log solve time of every candidate depth
        float feat[kNumCostDepths * kCostFeatures];
        for (int i = 0; i < kNumCostDepths; ++i)
            CKS(candidate_features(p, kCostDepths[i], feat + i * kCostFeatures, s));
        float pred[kNumCostDepths];
        CKS(costmodel_predict(net, feat, kNumCostDepths, pred, s));
        int best = 0;
        for (int i = 1; i < kNumCostDepths; ++i)
            if (pred[i] < pred[best]) best = i;
        p->chosen_depth = kCostDepths[best];
        if (kCostDepths[best] >= kThinOnly) {
            tau = kThinRows;
            d_max = kCostDepths[best] - kThinOnly;
            rho = kThinBudget;
        } else {
            tau = INT64_MAX;
            d_max = kCostDepths[best];
            rho = INFINITY;
        }
    } else if (prm.select_mode == SPTRSV_SELECT_SEGMODEL && default_segmodel()) {
        std::vector<std::pair<int32_t, int32_t>> segs;
        // the network was trained on segments of depth <= kSegMaxDepth
        CKS(segmodel_segments(p, default_segmodel(),
                              std::min(std::max(prm.max_depth, 0), kSegMaxDepth), s, &segs));
        for (auto &sg : segs) {
            p->seg_first.push_back(sg.first);
            p->seg_depth.push_back(sg.second);
        }
        return SPTRSV_OK;
    } else if (prm.select_mode == SPTRSV_SELECT_CRITPATH ||
               prm.select_mode == SPTRSV_SELECT_SEGMODEL) {
        // (SELECT_SEGMODEL without a network: the critical-path selection)
        std::vector<std::pair<int32_t, int32_t>> segs;
        CKS(critpath_segments(p, prm.hop_weight > 0 ? prm.hop_weight : 16, prm.max_depth, s,
                              &segs));
        for (auto &sg : segs) {
            p->seg_first.push_back(sg.first);
            p->seg_depth.push_back(sg.second);
        }
        return SPTRSV_OK;
    } else if (prm.select_mode == SPTRSV_SELECT_FIXED) {
        tau = INT64_MAX;
        d_max = prm.depth;
        rho = INFINITY;
    } else if (prm.select_mode == SPTRSV_SELECT_HEURISTIC ||
               prm.select_mode == SPTRSV_SELECT_COSTMODEL) {
        // heuristic H, also the fallback when no cost model is attached
        tau = prm.thin_rows;
        d_max = prm.max_depth;
        rho = prm.flop_budget;
    } else {
        return SPTRSV_ERR_UNSUPPORTED;
    }
    std::vector<std::pair<int32_t, int32_t>> segs;
    int64_t added = 0;
    if (d_max == 0) {
        for (int32_t l = 0; l < nlev; ++l) segs.emplace_back(l, 0);
    } else {
        CKS(compute_segments(p, tau, d_max, rho, s, &segs, &added));
    }
    for (auto &sg : segs) {
        p->seg_first.push_back(sg.first);
        p->seg_depth.push_back(sg.second);
    }
    return SPTRSV_OK;
}

// Rewritten rows of the chosen segments, computed on the device.
sptrsv_status_t build_rewritten(sptrsv_plan_t p, cudaStream_t s) {
    p->rw_off.reset();
    p->rw_col.reset();
    p->rw_val.reset();
    p->rw_nb.reset();
    p->pos_item.reset();
    p->nitems = 0;
    p->rows_rewritten = 0;
    std::vector<int32_t> ql, qt;
    std::vector<int64_t> qoff(1, 0);
    for (size_t i = 0; i < p->seg_first.size(); ++i) {
        const int32_t t = p->seg_first[i], d = p->seg_depth[i];
        for (int32_t l = t + 1; l <= t + d; ++l) {
            ql.push_back(l);
            qt.push_back(t);
            qoff.push_back(qoff.back() + (p->h_level_ptr[l + 1] - p->h_level_ptr[l]));
        }
    }
    const int64_t nitems = qoff.back();
    if (nitems == 0) return SPTRSV_OK;
    const int32_t nq = (int32_t)ql.size();
    DevArr<int32_t> d_ql, d_qt, irow, itgt, ipos, fill;
    DevArr<int64_t> d_qoff, stmp;
    CK(upload(d_ql, ql, s));
    CK(upload(d_qt, qt, s));
    CK(upload(d_qoff, qoff, s));
    CK(irow.alloc(nitems));
    CK(itgt.alloc(nitems));
    CK(ipos.alloc(nitems));
    CK(fill.alloc(nitems));
    CK(launch_expand_queries(nq, d_ql.p, d_qt.p, d_qoff.p, p->level_ptr.p, p->perm.p, irow.p,
                             itgt.p, nullptr, ipos.p, s));
    const int cap = p->prm.max_row_fill;
    CK(launch_rewrite_count(nitems, irow.p, itgt.p, nullptr, p->row_ptr.p, p->col.p, p->level.p,
                            cap, fill.p, nullptr, nullptr, nullptr, p->num_sms, s));
    CK(p->rw_off.alloc(nitems + 1));
    CK(stmp.alloc(scan_tmp_elems(nitems)));
    CK(exclusive_scan_i32_i64(fill.p, p->rw_off.p, nitems, stmp.p, s));
    int64_t total = 0;
    CK(cudaMemcpyAsync(&total, p->rw_off.p + nitems, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (total < 0 || total > INT32_MAX) return SPTRSV_ERR_UNSUPPORTED;
    CK(p->rw_col.alloc(total));
    CK(p->rw_val.alloc(total));
    CK(p->rw_nb.alloc(nitems));
    CK(launch_rewrite_numeric(nitems, irow.p, itgt.p, p->rw_off.p, p->row_ptr.p, p->col.p,
                              p->val.p, p->level.p, cap, p->rw_col.p, p->rw_val.p, p->rw_nb.p,
                              p->status.p, p->num_sms, s));
    CK(p->pos_item.alloc(p->n));
    CK(launch_pos_item(p->n, nitems, ipos.p, p->pos_item.p, s));
    CKS(sync_status(p, s));
    p->nitems = nitems;
    p->rows_rewritten = (int32_t)nitems;
    return SPTRSV_OK;
}

// Level-ordered solve structure for layout L.
template <typename T>
sptrsv_status_t build_struct(sptrsv_plan_t p, SolveStruct<T> &ss, int L, cudaStream_t s) {
    const int H = 32 / L;
    const int32_t nseg = (int32_t)p->seg_first.size();
    std::vector<int32_t> c_row0, c_nrows, lvl_chunk(nseg + 1, 0);
    for (int32_t sg = 0; sg < nseg; ++sg) {
        const int32_t t = p->seg_first[sg], d = p->seg_depth[sg];
        const int32_t a = p->h_level_ptr[t], b = p->h_level_ptr[t + d + 1];
        for (int32_t r = a; r < b; r += H) {
            c_row0.push_back(r);
            c_nrows.push_back(std::min<int32_t>(H, b - r));
        }
        lvl_chunk[sg + 1] = (int32_t)c_row0.size();
    }
    const int32_t nchunks = (int32_t)c_row0.size();
    DevArr<int32_t> d_row0, d_nrows, d_width;
    DevArr<int64_t> d_slots, d_off, stmp;
    CK(upload(d_row0, c_row0, s));
    CK(upload(d_nrows, c_nrows, s));
    CK(upload(ss.lvl_chunk, lvl_chunk, s));
    CK(d_width.alloc(nchunks));
    CK(d_slots.alloc(nchunks));
    CK(d_off.alloc((size_t)nchunks + 1));
    CK(stmp.alloc(scan_tmp_elems(nchunks)));
    const int32_t *pos_item = p->nitems > 0 ? p->pos_item.p : nullptr;
    CK(launch_chunk_width(nchunks, d_row0.p, d_nrows.p, L, p->perm.p, p->offdeg.p, pos_item,
                          p->rw_off.p, d_slots.p, d_width.p, s));
    CK(exclusive_scan_i64_i64(d_slots.p, d_off.p, nchunks, stmp.p, s));
    int64_t total = 0;
    CK(cudaMemcpyAsync(&total, d_off.p + nchunks, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (total > INT32_MAX) return SPTRSV_ERR_UNSUPPORTED;
    // chunk widths: the staging width that covers 99% of the chunks
    {
        std::vector<int32_t> wd(nchunks);
        CK(cudaMemcpyAsync(wd.data(), d_width.p, nchunks * sizeof(int32_t),
                           cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        std::vector<int64_t> hist(kStageZMax + 2, 0);
        for (int32_t w : wd) ++hist[std::min<int32_t>(w, kStageZMax + 1)];
        int64_t acc = 0;
        ss.width_p99 = kStageZMax + 1;
        for (int z = 0; z <= kStageZMax; ++z) {
            acc += hist[z];
            if (acc * 100 >= (int64_t)nchunks * 99) {
                ss.width_p99 = z;
                break;
            }
        }
    }
    CK(ss.meta.alloc(nchunks));
    // every chunk starts on a multiple of 4 entries and the arrays are
    // zeroed, so the staged solve copies whole 16-byte units; row_id and
    // diag hold a few spare elements for the same reason
    CK(ss.ecol.alloc(total));
    CK(ss.eval.alloc(total));
    CK(cudaMemsetAsync(ss.ecol.p, 0, (size_t)total * sizeof(int32_t), s));
    CK(cudaMemsetAsync(ss.eval.p, 0, (size_t)total * sizeof(T), s));
    CK(ss.row_id.alloc((size_t)p->n + 4));
    CK(ss.diag.alloc(2 * ((size_t)p->n + 4)));
    CK(cudaMemsetAsync(ss.row_id.p + p->n, 0, 4 * sizeof(int32_t), s));
    CK(cudaMemsetAsync(ss.diag.p + 2 * (size_t)p->n, 0, 8 * sizeof(T), s));
    CK(launch_chunk_fill<T>(nchunks, L, d_row0.p, d_nrows.p, d_width.p, d_off.p, p->perm.p,
                            p->row_ptr.p, p->col.p, p->val.p, pos_item, p->rw_off.p,
                            p->rw_col.p, p->rw_val.p, ss.meta.p, ss.ecol.p, ss.eval.p,
                            ss.row_id.p, ss.diag.p, s));
    CK(ss.chunk_level.alloc(nchunks));
    CK(launch_chunk_level(nseg, ss.lvl_chunk.p, ss.chunk_level.p, s));
    if (p->rev) CK(launch_struct_reverse(p->n, ss.row_id.p, total, ss.ecol.p, s));
    CK(cudaStreamSynchronize(s));
    ss.n = p->n;
    ss.nlev = nseg;
    ss.nchunks = nchunks;
    ss.h_lvl_chunk = std::move(lvl_chunk);
    ss.sched_nw = 0;
    ss.blob_valid = false;
    ss.run_encoded = -1;
    ss.run_slots = 0;
    ss.L = L;
    ss.nslots = total;
    ss.built = true;
    if ((const void *)&ss == (const void *)&p->s64) p->tail = TailStruct{};   // records of the old one
    return SPTRSV_OK;
}

// Phases of the barrier kernel: maximal runs (>= 2) of consecutive levels of
// at most run_rows rows become one CTA-local phase, each holding at most
// kMaxRunSlots rows in total (its unknowns live in shared memory); the run
// chunks' x terms that read rows of the same run are then encoded as
// shared-memory slots.
constexpr int32_t kMaxRunSlots = 8192;

template <typename T>
sptrsv_status_t build_phases(sptrsv_plan_t p, SolveStruct<T> &ss, int run_rows, cudaStream_t s) {
    std::vector<int2> ph;
    const int32_t nseg = (int32_t)p->seg_first.size();
    auto seg_rows = [&](int32_t sg) {
        const int32_t t = p->seg_first[sg], d = p->seg_depth[sg];
        return p->h_level_ptr[t + d + 1] - p->h_level_ptr[t];
    };
    int32_t sg = 0;
    while (sg < nseg) {
        if (run_rows > 0 && seg_rows(sg) <= run_rows) {
            // runs are capped so that the CTAs waiting at the next grid
            // barrier never wait longer than a fraction of the wait bound
            constexpr int32_t kMaxRunLevels = 16384;
            int32_t e = sg;
            int64_t rows = 0;
            while (e < nseg && e - sg < kMaxRunLevels && seg_rows(e) <= run_rows &&
                   rows + seg_rows(e) <= kMaxRunSlots) {
                rows += seg_rows(e);
                ++e;
            }
            if (e - sg >= 2) {
                ph.push_back(make_int2(sg, -e));
                sg = e;
                continue;
            }
        }
        ph.push_back(make_int2(sg, sg + 1));
        ++sg;
    }
    CK(upload(ss.phases, ph, s));
    ss.nphases = (int32_t)ph.size();
    // shared-memory slots for the unknowns of each run
    std::vector<int32_t> run_chunk;
    std::vector<int2> run_span;
    std::vector<int32_t> lvl_chunk(nseg + 1);
    CK(cudaMemcpy(lvl_chunk.data(), ss.lvl_chunk.p, (nseg + 1) * sizeof(int32_t),
                  cudaMemcpyDeviceToHost));
    int32_t slots = 0;
    for (const int2 &q : ph) {
        if (q.y > 0) continue;
        const int32_t l0 = q.x, l1 = -q.y;
        const int32_t P0 = p->h_level_ptr[p->seg_first[l0]];
        const int32_t P1 = p->h_level_ptr[p->seg_first[l1 - 1] + p->seg_depth[l1 - 1] + 1];
        slots = std::max(slots, P1 - P0);
        for (int32_t c = lvl_chunk[l0]; c < lvl_chunk[l1]; ++c) {
            run_chunk.push_back(c);
            run_span.push_back(make_int2(P0, P1));
        }
    }
    ss.run_slots = slots;
    {
        std::vector<int32_t> p0(ss.nchunks, -1);
        for (size_t i = 0; i < run_chunk.size(); ++i) p0[run_chunk[i]] = run_span[i].x;
        CK(upload(ss.chunk_run_p0, p0, s));
    }
    if (!run_chunk.empty()) {
        DevArr<int32_t> d_rc, pos;
        DevArr<int2> d_rs;
        CK(upload(d_rc, run_chunk, s));
        CK(upload(d_rs, run_span, s));
        CK(pos.alloc(p->n));
        CK(launch_encode_runs(p->n, ss.L, ss.row_id.p, ss.meta.p, (int32_t)run_chunk.size(),
                              d_rc.p, d_rs.p, pos.p, ss.ecol.p, s));
        CK(cudaStreamSynchronize(s));
        ss.blob_valid = false;   // the entries changed
    }
    CK(cudaStreamSynchronize(s));
    ss.run_encoded = run_rows;
    return SPTRSV_OK;
}

int auto_lanes(sptrsv_plan_t p) {
    int64_t len = 0;
    // average off-diagonal terms per row of the structure about to be built
    len = (p->nnz - p->n);
    if (p->nitems > 0) len += (p->nnz_x + p->nnz_b) - (p->nnz - p->n);
    const double avg = p->n ? (double)len / p->n : 0.0;
    if (avg <= 16) return 1;
    if (avg <= 32) return 2;
    if (avg <= 64) return 4;
    return 8;
}

// Staging width of the synchronisation-free one-column solve over ss (0 =
// not staged): the requested or 99% width, capped so that the slots of
// kStageWarpsPerSM warps fit an SM's shared memory (the staged kernel's
// registers allow about 20 resident warps per SM).
template <typename T>
int stage_width(sptrsv_plan_t p, const SolveStruct<T> &ss) {
    const SolveConfig &c = p->cfg;
    if (!c.syncfree || c.stage_off || p->prm.stage_z < 0 || !ss.built) return 0;
    int z = p->prm.stage_z > 0 ? p->prm.stage_z : ss.width_p99;
    z = std::min(z, stage_cap_z<T>(ss.L, p->smem_per_sm, kStageWarpsPerSM));
    return std::max(z, 0);
}

int grid_for(sptrsv_plan_t p, int nr, bool f32) {
    const SolveConfig &c = p->cfg;
    const int mx =
        f32 ? max_coresident_ctas<float>(c.L, nr, c.syncfree, c.block_threads, p->num_sms,
                                         p->s32.run_slots, nr == 1 ? stage_width(p, p->s32) : 0)
            : max_coresident_ctas<double>(c.L, nr, c.syncfree, c.block_threads, p->num_sms,
                                          p->s64.run_slots, nr == 1 ? stage_width(p, p->s64) : 0);
    if (mx <= 0) return 0;
    int g = c.grid > 0 ? c.grid : mx;
    return std::min(g, mx);
}

// Count x and b terms of the solve structure (the info fields nnz_x/nnz_b).
sptrsv_status_t count_terms(sptrsv_plan_t p, cudaStream_t s) {
    const int32_t n = p->n;
    if (n == 0) {
        p->nnz_x = p->nnz_b = 0;
        return SPTRSV_OK;
    }
    DevArr<int64_t> xc, bc, xs, bs, tmp;
    CK(xc.alloc(n));
    CK(bc.alloc(n));
    CK(xs.alloc(n + 1));
    CK(bs.alloc(n + 1));
    CK(tmp.alloc(scan_tmp_elems(n)));
    CK(launch_export_count(p->s64.nchunks, p->s64.L, p->s64.meta.p, p->s64.ecol.p,
                           p->s64.row_id.p, p->n, xc.p, bc.p, s));
    CK(exclusive_scan_i64_i64(xc.p, xs.p, n, tmp.p, s));
    CK(exclusive_scan_i64_i64(bc.p, bs.p, n, tmp.p, s));
    CK(cudaMemcpyAsync(&p->nnz_x, xs.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&p->nnz_b, bs.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return SPTRSV_OK;
}

// Records of the single-CTA tail for width limit `rows`.  The tail is the
// longest suffix of new levels with at most `rows` rows each (none when
// shorter than kMinTailLevels levels), cut into segments where the level
// width crosses kTailThinRows for good (both sides at least kMinSegLevels
// levels): each segment is solved by one CTA after a fold pass, so a
// segment's rows carry only the terms of its own unknowns.  Segments are
// taken from the last one back; a row with more than 16 such terms splits
// its segment around its level (at most kMaxTailSegs segments).
constexpr int32_t kMinTailLevels = 8;
constexpr int32_t kMinSegLevels = 64;
constexpr int32_t kMaxTailSegs = 64;
constexpr int32_t kTailThinRows = 32;
constexpr int32_t kTailWindow = 16384;   // shared-memory window of unknowns (128 KiB)

sptrsv_status_t build_tail(sptrsv_plan_t p, int rows, cudaStream_t s) {
    TailStruct &t = p->tail;
    t = TailStruct{};
    t.for_rows = rows;
    t.built = true;
    const SolveStruct<double> &ss = p->s64;
    const int32_t nseg = (int32_t)p->seg_first.size();
    auto lo = [&](int32_t g) { return p->h_level_ptr[p->seg_first[g]]; };
    auto hi = [&](int32_t g) {
        return p->h_level_ptr[p->seg_first[g] + p->seg_depth[g] + 1];
    };
    int32_t g0 = nseg;
    while (g0 > 0 && hi(g0 - 1) - lo(g0 - 1) <= rows) --g0;
    if (nseg - g0 < kMinTailLevels || !ss.built || ss.run_encoded > 0) return SPTRSV_OK;
    // cuts where the width class changes and stays changed
    std::vector<int32_t> thin_before(nseg - g0 + 1, 0);
    for (int32_t g = g0; g < nseg; ++g)
        thin_before[g - g0 + 1] = thin_before[g - g0] + (hi(g) - lo(g) < kTailThinRows);
    auto thin_in = [&](int32_t a, int32_t b) { return thin_before[b - g0] - thin_before[a - g0]; };
    std::vector<int32_t> cuts{g0};
    bool cls = hi(g0) - lo(g0) < kTailThinRows;
    for (int32_t g = g0 + 1; g + kMinSegLevels <= nseg; ++g) {
        const bool c = hi(g) - lo(g) < kTailThinRows;
        if (c == cls || g - cuts.back() < kMinSegLevels) continue;
        const int32_t nthin = thin_in(g, g + kMinSegLevels);
        if (c ? nthin == kMinSegLevels : nthin == 0) {
            cuts.push_back(g);
            cls = c;
        }
    }
    cuts.push_back(nseg);
    const std::vector<int32_t> &lc = ss.h_lvl_chunk;
    DevArr<int32_t> pos_of, flags;
    CK(pos_of.alloc(p->n));
    CK(flags.alloc(2));
    CK(launch_pos_of_row(p->n, ss.row_id.p, pos_of.p, s));
    // ranges still to build, the last one on top; a range whose rows have
    // more than 16 in-segment terms is split around its last level holding
    // such a row (alone, that level is a segment without in-segment terms:
    // rows of one level never read each other), and the rest recounted
    std::vector<std::pair<int32_t, int32_t>> todo;
    for (size_t j = 0; j + 1 < cuts.size(); ++j) todo.emplace_back(cuts[j], cuts[j + 1]);
    std::vector<TailSeg> segs;   // last first
    while (!todo.empty()) {
        const int32_t ga = todo.back().first, gb = todo.back().second;
        todo.pop_back();
        const int32_t P0 = lo(ga), P1 = gb < nseg ? lo(gb) : p->n;
        const int32_t nr = P1 - P0, nl = gb - ga;
        const int32_t c0 = lc[ga], c1 = gb < nseg ? lc[gb] : ss.nchunks;
        int32_t maxw = 0;
        for (int32_t g = ga; g < gb; ++g) maxw = std::max(maxw, hi(g) - lo(g));
        TailSeg sg;
        std::vector<int32_t> tlp(nl + 1);
        for (int32_t g = 0; g < nl; ++g) tlp[g] = lo(ga + g) - P0;
        tlp[nl] = nr;
        DevArr<int32_t> cnt_a, cnt_n;
        DevArr<int64_t> tmp;
        CK(upload(sg.lp, tlp, s));
        CK(cnt_a.alloc(nr));
        CK(cnt_n.alloc(nr));
        CK(sg.aptr.alloc((size_t)nr + 1));
        CK(tmp.alloc(scan_tmp_elems(nr)));
        CK(cudaMemsetAsync(flags.p, 0, 2 * sizeof(int32_t), s));
        CK(launch_tail_count(c0, c1, ss.L, p->n, ss.meta.p, ss.ecol.p, pos_of.p, P0, cnt_a.p,
                             cnt_n.p, flags.p, flags.p + 1, s));
        CK(exclusive_scan_i32_i64(cnt_a.p, sg.aptr.p, nr, tmp.p, s));
        int32_t hflags[2] = {0, 0};
        int64_t na = 0;
        CK(cudaMemcpyAsync(hflags, flags.p, sizeof(hflags), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&na, sg.aptr.p + nr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (hflags[1] != 0) break;   // run slots: this segment and those before, no tail
        if (hflags[0] > 16) {
            if (segs.size() + todo.size() + 3 > (size_t)kMaxTailSegs) break;
            std::vector<int32_t> hn(nr);
            CK(cudaMemcpy(hn.data(), cnt_n.p, sizeof(int32_t) * nr, cudaMemcpyDeviceToHost));
            int32_t plast = nr - 1;
            while (hn[plast] <= 16) --plast;
            int32_t gs = ga;   // the level holding position plast
            while (gs + 1 < gb && lo(gs + 1) - P0 <= plast) ++gs;
            if (gs > ga) todo.emplace_back(ga, gs);
            todo.emplace_back(gs, gs + 1);
            if (gs + 1 < gb) todo.emplace_back(gs + 1, gb);
            continue;
        }
        const int32_t K = hflags[0] <= 4 ? 4 : hflags[0] <= 8 ? 8 : 16;
        const int32_t T = std::max(32, (maxw + 31) / 32 * 32);
        CK(sg.row.alloc(nr));
        CK(sg.nn.alloc(nr));
        CK(sg.diag.alloc(nr));
        CK(sg.term.alloc((size_t)K * nr));
        CK(sg.acol.alloc(na > 0 ? na : 1));
        CK(sg.aval.alloc(na > 0 ? na : 1));
        CK(sg.s0.alloc(nr));
        CK(launch_tail_fill(c0, c1, ss.L, p->n, ss.meta.p, ss.ecol.p, ss.eval.p, ss.row_id.p,
                            ss.diag.p, ss.chunk_level.p, ga, sg.lp.p, pos_of.p, P0, kTailWindow,
                            T, K, nr, sg.aptr.p, sg.row.p, sg.diag.p, sg.nn.p, sg.term.p,
                            sg.acol.p, sg.aval.p, s));
        CK(cudaStreamSynchronize(s));
        sg.lev0 = ga;
        sg.c0 = c0;
        sg.P0 = P0;
        sg.nrows = nr;
        sg.nlev = nl;
        sg.K = K;
        sg.T = T;
        sg.W = kTailWindow;
        segs.push_back(std::move(sg));
    }
    if (segs.empty()) return SPTRSV_OK;
    std::reverse(segs.begin(), segs.end());
    t.lev0 = segs.front().lev0;
    t.c0 = segs.front().c0;
    for (const TailSeg &sg : segs) t.nlev += sg.nlev;
    t.segs = std::move(segs);
    return SPTRSV_OK;
}


// Level-major chunk schedule of the synchronisation-free kernels for nw
// warps, the autotuner's alternative to dealing the chunk list round robin:
// each level's chunks are dealt to warps 0, 1, 2, ... in turn, and a warp
// takes its chunks level by level, so that a warp holds about one chunk per
// level of a wide matrix instead of one every few levels.  (On the 128^3
// stencil it measured slower than round robin, 0.51 against 0.46 ms at depth
// 2: every warp then polls the same level at once, which loads the L2.)
template <typename T>
sptrsv_status_t build_sched(SolveStruct<T> &ss, int32_t nw, cudaStream_t s) {
    if (nw <= 0 || !ss.built || ss.nchunks == 0) return SPTRSV_OK;
    if (ss.sched_nw == nw && ss.sched.p) return SPTRSV_OK;
    const std::vector<int32_t> &lc = ss.h_lvl_chunk;
    std::vector<int32_t> ptr((size_t)nw + 1, 0), sched((size_t)ss.nchunks);
    for (size_t l = 0; l + 1 < lc.size(); ++l)
        for (int32_t i = 0; i < lc[l + 1] - lc[l]; ++i) ++ptr[(size_t)(i % nw) + 1];
    for (int32_t w = 0; w < nw; ++w) ptr[(size_t)w + 1] += ptr[w];
    std::vector<int32_t> pos(ptr.begin(), ptr.end() - 1);
    for (size_t l = 0; l + 1 < lc.size(); ++l)
        for (int32_t i = 0; i < lc[l + 1] - lc[l]; ++i) sched[pos[i % nw]++] = lc[l] + i;
    CK(upload(ss.sched, sched, s));
    CK(upload(ss.sched_ptr, ptr, s));
    CK(cudaStreamSynchronize(s));
    ss.sched_nw = nw;
    return SPTRSV_OK;
}

// Chunk blobs of the staged kernels: every chunk once more as one
// contiguous run of 16-byte units (BlobLayout), built from the entries.
template <typename T>
sptrsv_status_t build_blob(SolveStruct<T> &ss, cudaStream_t s) {
    if (!ss.built || ss.blob_valid || ss.nchunks == 0) return SPTRSV_OK;
    DevArr<int64_t> units, tmp;
    CK(units.alloc(ss.nchunks));
    CK(ss.bofs.alloc((size_t)ss.nchunks + 1));
    CK(tmp.alloc(scan_tmp_elems(ss.nchunks)));
    CK(launch_blob_units<T>(ss.nchunks, ss.L, ss.meta.p, units.p, s));
    CK(exclusive_scan_i64_i64(units.p, ss.bofs.p, ss.nchunks, tmp.p, s));
    int64_t total = 0;
    CK(cudaMemcpyAsync(&total, ss.bofs.p + ss.nchunks, sizeof(int64_t), cudaMemcpyDeviceToHost,
                       s));
    CK(cudaStreamSynchronize(s));
    CK(ss.blob.alloc((size_t)total));
    CK(cudaMemsetAsync(ss.blob.p, 0, (size_t)total * sizeof(uint4), s));
    CK(launch_blob_fill<T>(ss.nchunks, ss.L, ss.meta.p, ss.row_id.p, ss.diag.p, ss.ecol.p,
                           ss.eval.p, ss.bofs.p, ss.blob.p, s));
    CK(cudaStreamSynchronize(s));
    ss.blob_valid = true;
    return SPTRSV_OK;
}

sptrsv_status_t apply_config(sptrsv_plan_t p, cudaStream_t s) {
    const bool f32 = p->prm.precision == SPTRSV_F32_IR;
    // run slots are encoded into the entries: a new run threshold needs a
    // freshly assembled structure
    const int runs = p->cfg.syncfree ? 0 : p->cfg.cta_run_rows;
    if (p->s64.L != p->cfg.L || !p->s64.built ||
        (p->s64.run_encoded > 0 && p->s64.run_encoded != runs))
        CKS(build_struct<double>(p, p->s64, p->cfg.L, s));
    if (p->s64.run_encoded != runs) CKS(build_phases<double>(p, p->s64, runs, s));
    if (f32) {
        if (p->s32.L != p->cfg.L || !p->s32.built ||
            (p->s32.run_encoded > 0 && p->s32.run_encoded != runs))
            CKS(build_struct<float>(p, p->s32, p->cfg.L, s));
        if (p->s32.run_encoded != runs) CKS(build_phases<float>(p, p->s32, runs, s));
    }
    if (!f32 && runs <= 0 && p->cfg.tail_rows > 0 && !p->injected &&
        (!p->tail.built || p->tail.for_rows != p->cfg.tail_rows))
        CKS(build_tail(p, p->cfg.tail_rows, s));
    // generated kernels for the tail's thin segments
    if (!f32 && p->tail.built && !p->tail.segs.empty() && p->prm.codegen_rows > 0 &&
        p->tail.gen_rows != p->prm.codegen_rows) {
        p->tail.gen_ms = 0;
        for (TailSeg &sg : p->tail.segs) {
            if (codegen_eligible(sg, p->prm.codegen_rows)) CKS(codegen_build(sg, p->tail.gen_ms));
            else sg.gen.reset();
        }
        p->tail.gen_rows = p->prm.codegen_rows;
    }
    // schedule and chunk blobs of the synchronisation-free kernels
    if (p->cfg.syncfree) {
        const int32_t nw = grid_for(p, 1, f32) * (p->cfg.block_threads / 32);
        if (p->cfg.sched_lm) {
            if (f32) CKS(build_sched(p->s32, nw, s));
            else CKS(build_sched(p->s64, nw, s));
        }
        if (f32 ? stage_width(p, p->s32) > 0 : stage_width(p, p->s64) > 0) {
            if (f32) CKS(build_blob(p->s32, s));
            else CKS(build_blob(p->s64, s));
        }
    }
    return SPTRSV_OK;
}

// The tail kernel takes over the trailing levels: one right-hand side, FP64,
// no CTA-local runs in the main kernel.
bool tail_active(sptrsv_plan_t p, int32_t nrhs) {
    const int runs = p->cfg.syncfree ? 0 : p->cfg.cta_run_rows;
    return !p->injected && nrhs == 1 && p->prm.precision != SPTRSV_F32_IR && runs <= 0 &&
           p->cfg.tail_rows > 0 && p->tail.built && p->tail.for_rows == p->cfg.tail_rows &&
           p->tail.nlev > 0;
}

sptrsv_status_t solve_impl(sptrsv_plan_t p, const double *b, double *x, int32_t nrhs,
                           cudaStream_t s);

// Times candidate launch configurations on the plan (median of a few solves)
// and keeps the fastest.  Stage 1 crosses lanes per row with the three
// execution modes (grid barrier, barrier + CTA-local runs, synchronisation
// free) at three launch shapes; stage 2 sweeps the launch shape of the two
// best (lanes, mode) pairs; stage 3 the polling back-off of the sync-free
// kernel.  Trials of long solves use fewer repetitions.
// Autotuning results are kept per process, keyed by what decides them: the
// device, the plan's shape (rows, entries, level sizes, the chosen segments,
// terms of the rewritten structure) and every request that constrains the
// search.  A plan with the same key takes the cached launch without timing.
struct TuneKey {
    int device;
    int32_t n, precision, nrhs_hint, lanes, block, grid, runs, backoff, tail, stage;
    int64_t nnz, nnz_x, nnz_b;
    uint64_t shape;
    bool operator<(const TuneKey &o) const {
        return std::tie(device, n, precision, nrhs_hint, lanes, block, grid, runs, backoff, tail,
                        stage, nnz, nnz_x, nnz_b, shape) <
               std::tie(o.device, o.n, o.precision, o.nrhs_hint, o.lanes, o.block, o.grid,
                        o.runs, o.backoff, o.tail, o.stage, o.nnz, o.nnz_x, o.nnz_b, o.shape);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, SolveConfig> g_tune_cache;

TuneKey tune_key(sptrsv_plan_t p) {
    uint64_t h = 1469598103934665603ull;  // FNV-1a over level sizes and segments
    auto mix = [&](uint64_t v) {
        for (int b = 0; b < 8; ++b) {
            h ^= (v >> (8 * b)) & 0xff;
            h *= 1099511628211ull;
        }
    };
    for (int32_t v : p->h_level_ptr) mix((uint64_t)(uint32_t)v);
    for (size_t i = 0; i < p->seg_first.size(); ++i)
        mix(((uint64_t)(uint32_t)p->seg_first[i] << 32) | (uint32_t)p->seg_depth[i]);
    const auto &q = p->prm;
    return TuneKey{p->device, p->n, q.precision, q.nrhs_hint, q.lanes_per_row, q.block_threads,
                   q.grid_blocks, q.cta_run_rows, q.poll_backoff_ns, q.tail_rows, q.stage_z, p->nnz,
                   p->nnz_x, p->nnz_b, h};
}

sptrsv_status_t autotune_search(sptrsv_plan_t p, cudaStream_t s);

sptrsv_status_t autotune(sptrsv_plan_t p, cudaStream_t s) {
    if (p->n == 0) return SPTRSV_OK;
    const TuneKey key = tune_key(p);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            p->cfg = it->second;
            p->tuned_from_cache = true;
            return apply_config(p, s);
        }
    }
    p->tuned_from_cache = false;
    CKS(autotune_search(p, s));
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = p->cfg;
    return SPTRSV_OK;
}

sptrsv_status_t autotune_search(sptrsv_plan_t p, cudaStream_t s) {
    const int32_t n = p->n;
    if (n == 0) return SPTRSV_OK;
    const bool f32 = p->prm.precision == SPTRSV_F32_IR;
    const int nrt = p->prm.nrhs_hint;  // columns of the trial solves
    DevArr<double> b, x;
    CK(b.alloc((size_t)n * nrt));
    CK(x.alloc((size_t)n * nrt));
    std::vector<double> ones((size_t)n * nrt, 1.0);
    CK(cudaMemcpyAsync(b.p, ones.data(), ones.size() * sizeof(double), cudaMemcpyHostToDevice,
                       s));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int warm = 2, reps = 5;
    double best_ms = 1e30;
    auto time_cfg = [&](double *ms_out) -> sptrsv_status_t {
        CKS(apply_config(p, s));
        // the first warm-up is timed: a shape four times slower than the best
        // so far is dropped without further solves
        CK(cudaEventRecord(e0, s));
        CKS(solve_impl(p, b.p, x.p, nrt, s));
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        float first = 0;
        CK(cudaEventElapsedTime(&first, e0, e1));
        if (first > 4.0 * best_ms) {
            CKS(sync_status(p, s));
            *ms_out = first;
            return SPTRSV_OK;
        }
        for (int w = 1; w < warm; ++w) CKS(solve_impl(p, b.p, x.p, nrt, s));
        std::vector<float> t;
        for (int r = 0; r < reps; ++r) {
            CK(cudaEventRecord(e0, s));
            CKS(solve_impl(p, b.p, x.p, nrt, s));
            CK(cudaEventRecord(e1, s));
            CK(cudaEventSynchronize(e1));
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            t.push_back(ms);
        }
        CKS(sync_status(p, s));
        std::sort(t.begin(), t.end());
        *ms_out = t[t.size() / 2];
        return SPTRSV_OK;
    };
    struct Trial {
        SolveConfig c;
        double ms;
    };
    std::vector<Trial> tried;
    auto same = [](const SolveConfig &a, const SolveConfig &c) {
        return a.L == c.L && a.syncfree == c.syncfree && a.block_threads == c.block_threads &&
               a.grid == c.grid && a.cta_run_rows == c.cta_run_rows &&
               a.backoff_ns == c.backoff_ns && a.tail_rows == c.tail_rows &&
               a.stage_off == c.stage_off && a.sched_lm == c.sched_lm;
    };
    SolveConfig best = p->cfg;
    auto trial = [&](const SolveConfig &c, double *ms) -> sptrsv_status_t {
        for (const Trial &t : tried)
            if (same(t.c, c)) {
                *ms = t.ms;
                return SPTRSV_OK;
            }
        *ms = 1e30;
        p->cfg = c;
        const int gmax = grid_for(p, nrt, f32);
        if (gmax <= 0 || (c.grid > 0 && gmax < c.grid)) return SPTRSV_OK;  // not co-resident
        CKS(time_cfg(ms));
        tried.push_back({c, *ms});
        if (*ms < best_ms) {
            best_ms = *ms;
            best = c;
        }
        if (best_ms > 5.0) {  // long solves: fewer repetitions
            warm = 1;
            reps = 3;
        }
        return SPTRSV_OK;
    };
    const int bt_req = p->prm.block_threads;
    const int grid_req = p->prm.grid_blocks;
    const int backoff0 = p->prm.poll_backoff_ns > 0 ? p->prm.poll_backoff_ns : 0;
    auto shaped = [&](SolveConfig c, int bt, int per_sm) {
        c.block_threads = bt_req > 0 ? bt_req : bt;
        c.grid = grid_req > 0 ? grid_req : per_sm * p->num_sms;
        if (c.cta_run_rows > 0) c.cta_run_rows = c.block_threads / c.L;
        return c;
    };
    std::vector<int> lanes = {1, 2, 4};
    const int la = auto_lanes(p);
    if (la > 4) lanes.push_back(la);
    if (nrt > 1) lanes = {p->cfg.L};  // laid out for the hinted columns
    // stage 1: lanes x mode at three launch shapes
    struct Pair {
        SolveConfig c;
        double ms;
    };
    std::vector<Pair> pairs;
    for (int L : lanes) {
        if (p->prm.lanes_per_row > 0 && L != p->prm.lanes_per_row) continue;
        for (int mode = 0; mode < 3; ++mode) {
            if (p->prm.cta_run_rows < 0 && mode == 1) continue;
            SolveConfig c;
            c.L = L;
            c.syncfree = mode == 2;
            c.backoff_ns = backoff0;
            c.cta_run_rows = mode == 1 ? 1 : 0;  // set from the block size by shaped()
            double pm = 1e30;
            const std::pair<int, int> shapes[3] = {{128, 4}, {128, 8}, {512, 1}};
            for (const auto &sh : shapes) {
                double ms;
                CKS(trial(shaped(c, sh.first, sh.second), &ms));
                pm = std::min(pm, ms);
            }
            pairs.push_back({c, pm});
        }
    }
    std::sort(pairs.begin(), pairs.end(),
              [](const Pair &a, const Pair &c) { return a.ms < c.ms; });
    // stage 2: launch shape of the two best pairs
    for (size_t i = 0; i < pairs.size() && i < 2; ++i) {
        if (pairs[i].ms >= 1e30) break;
        for (int bt : {128, 256, 512})
            for (int per_sm : {1, 2, 4, 8}) {
                if (bt * per_sm > 2048) continue;
                double ms;
                CKS(trial(shaped(pairs[i].c, bt, per_sm), &ms));
            }
    }
    // stage 3: polling back-off of the synchronisation-free kernel
    if (best.syncfree && p->prm.poll_backoff_ns < 0) {
        const SolveConfig b0 = best;
        for (int ns : {32, 128, 512}) {
            SolveConfig c = b0;
            c.backoff_ns = ns;
            double ms;
            CKS(trial(c, &ms));
        }
    }
    // stage 3b: the synchronisation-free kernel with its chunks dealt
    // level-major instead of round robin, and without shared-memory staging
    if (best.syncfree) {
        SolveConfig c = best;
        c.sched_lm = true;
        double ms;
        CKS(trial(c, &ms));
    }
    if (best.syncfree && p->prm.stage_z == 0 && nrt == 1) {
        SolveConfig c = best;
        c.stage_off = true;
        double ms;
        CKS(trial(c, &ms));
    }
    // stage 4: the single-CTA tail over trailing levels of at most 32..256 rows
    if (!f32 && nrt == 1 && p->prm.tail_rows >= 0 &&
        (best.syncfree || best.cta_run_rows <= 0)) {
        const SolveConfig b0 = best;
        std::vector<int> widths = {32, 64, 128, 256};
        if (p->prm.tail_rows > 0) widths = {p->prm.tail_rows};
        for (int w : widths) {
            SolveConfig c = b0;
            c.tail_rows = w;
            double ms;
            CKS(trial(c, &ms));
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->cfg = best;
    return apply_config(p, s);
}

void resolve_params(sptrsv_plan_t p, const sptrsv_transform_params_t *in) {
    sptrsv_transform_params_t q = *in;
    if (q.thin_rows <= 0) q.thin_rows = std::max(1, p->num_sms * 64 / 4);
    if (q.max_depth <= 0) q.max_depth = q.max_depth == 0 ? 0 : 8;
    if (q.max_depth > 16) q.max_depth = 16;
    if (q.depth < 0) q.depth = 0;
    if (q.depth > 16) q.depth = 16;
    if (q.flop_budget < 0) q.flop_budget = 0.10;
    if (q.max_row_fill <= 0) q.max_row_fill = 1024;
    if (q.max_row_fill > 4096) q.max_row_fill = 4096;
    if (q.ir_tol <= 0) q.ir_tol = 1e-15;
    if (q.ir_max_iter < 0) q.ir_max_iter = 8;
    if (q.ir_max_iter > 64) q.ir_max_iter = 64;
    if (q.wait_timeout_ms <= 0) q.wait_timeout_ms = 5000;
    if (q.nrhs_hint < 1) q.nrhs_hint = 1;
    if (q.nrhs_hint > 32) q.nrhs_hint = 32;
    if (q.tail_rows > 256) q.tail_rows = 256;
    if (q.codegen_rows < 0) q.codegen_rows = 0;
    if (q.codegen_rows > kCodegenMaxRows) q.codegen_rows = kCodegenMaxRows;
    if (q.stage_z > kStageZMax) q.stage_z = kStageZMax;
    p->prm = q;
    p->thin_rows_used = q.thin_rows;
}

sptrsv_status_t ensure_ir(sptrsv_plan_t p, int64_t count) {
    if ((int64_t)p->d32.n < count) CK(p->d32.alloc(count));
    if ((int64_t)p->r64.n < count) CK(p->r64.alloc(count));
    return SPTRSV_OK;
}

sptrsv_status_t solve_impl(sptrsv_plan_t p, const double *b, double *x, int32_t nrhs,
                           cudaStream_t s) {
    const int32_t n = p->n;
    const uint64_t tmo = timeout_ns(p);
    if (p->prm.precision != SPTRSV_F32_IR) {
        SolveData<double> sd = p->s64.view();
        sd.backoff_ns = p->cfg.backoff_ns;
        sd.stage_z = stage_width(p, p->s64);
        if (!p->cfg.sched_lm) sd.sched = nullptr;
        if (p->profiling) CK(cudaEventRecord(p->prof_ev[0], s));
        if (tail_active(p, nrhs)) {
            const TailStruct &t = p->tail;
            if (t.c0 > 0) {
                SolveData<double> sm = sd;
                sm.nchunks = t.c0;     // the synchronisation-free kernel's chunks
                sm.nphases = t.lev0;   // the barrier kernel's phases: one per level
                LaunchCfg lc{p->cfg.block_threads, grid_for(p, 1, false)};
                if (lc.grid <= 0) return SPTRSV_ERR_CUDA;
                CK(launch_solve<double>(sm, b, x, n, 1, 1, p->cfg.syncfree, lc, p->status.p, tmo,
                                        false, s));
            }
            for (const TailSeg &sg : t.segs) {
                if (sg.gen.fn && t.gen_rows == p->prm.codegen_rows) CK(codegen_launch(sg, b, x, s));
                else CK(launch_tail(tail_view(sg), b, x, sg.T, s));
            }
            if (p->profiling) {
                CK(cudaEventRecord(p->prof_ev[1], s));
                p->prof_valid = true;
            }
            return SPTRSV_OK;
        }
        for (int32_t c0 = 0; c0 < nrhs; c0 += 32) {
            const int nr = std::min<int32_t>(32, nrhs - c0);
            LaunchCfg lc{p->cfg.block_threads, grid_for(p, nr, false)};
            if (lc.grid <= 0) return SPTRSV_ERR_CUDA;
            CK(launch_solve<double>(sd, b + c0, x + c0, n, nrhs, nr, p->cfg.syncfree, lc,
                                    p->status.p, tmo, false, s));
        }
        if (p->profiling) {
            CK(cudaEventRecord(p->prof_ev[1], s));
            p->prof_valid = true;
        }
        return SPTRSV_OK;
    }
    p->prof_valid = false;
    // FP32 solve with FP64 iterative refinement
    const int64_t count = (int64_t)n * nrhs;
    CKS(ensure_ir(p, count));
    SolveData<float> sd = p->s32.view();
    sd.backoff_ns = p->cfg.backoff_ns;
    sd.stage_z = stage_width(p, p->s32);
    if (!p->cfg.sched_lm) sd.sched = nullptr;
    auto solve32 = [&](const double *rhs, bool skip) -> sptrsv_status_t {
        for (int32_t c0 = 0; c0 < nrhs; c0 += 32) {
            const int nr = std::min<int32_t>(32, nrhs - c0);
            LaunchCfg lc{p->cfg.block_threads, grid_for(p, nr, true)};
            if (lc.grid <= 0) return SPTRSV_ERR_CUDA;
            CK(launch_solve<float>(sd, rhs + c0, p->d32.p + c0, n, nrhs, nr, p->cfg.syncfree,
                                   lc, p->status.p, tmo, skip, s));
        }
        return SPTRSV_OK;
    };
    CK(launch_ir_begin(p->status.p, b, count, s));
    CKS(solve32(b, false));
    CK(launch_ir_update(x, p->d32.p, count, true, p->status.p, s));
    for (int it = 0; it < p->prm.ir_max_iter; ++it) {
        CK(launch_residual(n, p->row_ptr.p, p->col.p, p->val.p, p->rev, b, x, p->r64.p, nrhs, nrhs,
                           p->status.p, s));
        CK(launch_ir_decide(p->status.p, p->prm.ir_tol, p->lnorm.p, s));
        CKS(solve32(p->r64.p, true));
        CK(launch_ir_update(x, p->d32.p, count, false, p->status.p, s));
    }
    return SPTRSV_OK;
}

// SPTRSV_SELECT_AUTO: every candidate rewrite is built and timed on the plan
// (synchronisation-free kernel, 1 and 4 lanes per row), and the fastest one
// is transformed with the caller's launch parameters.
sptrsv_status_t select_auto(sptrsv_plan_t p, const sptrsv_transform_params_t *prm,
                            sptrsv_stream_t stream) {
    const double t0 = now_ms();
    cudaStream_t s = (cudaStream_t)stream;
    struct Cand {
        int code;
        sptrsv_transform_params_t q;
    };
    std::vector<Cand> cands;
    auto add = [&](int code, int mode, int depth, int thin, int dmax, double rho) {
        for (const Cand &c : cands)
            if (c.code == code) return;
        sptrsv_transform_params_t q = *prm;
        q.select_mode = mode;
        q.depth = depth;
        if (mode == SPTRSV_SELECT_HEURISTIC) {
            q.thin_rows = thin;
            q.max_depth = dmax;
            q.flop_budget = rho;
        }
        cands.push_back({code, q});
    };
    add(0, SPTRSV_SELECT_NONE, 0, 0, 0, 0);
    for (int d = 1; d <= 3; ++d) add(d, SPTRSV_SELECT_FIXED, d, 0, 0, 0);
    add(200, SPTRSV_SELECT_HEURISTIC, 0, prm->thin_rows, prm->max_depth, prm->flop_budget);
    add(kThinOnly + 8, SPTRSV_SELECT_HEURISTIC, 0, kThinRows, 8, kThinBudget);
    add(kThinOnly + 16, SPTRSV_SELECT_HEURISTIC, 0, kThinRows, 16, kThinBudget);
    {   // the critical-path selection, at most 4 levels per segment
        sptrsv_transform_params_t q = *prm;
        q.select_mode = SPTRSV_SELECT_CRITPATH;
        q.max_depth = std::min(std::max(prm->max_depth, 1), 4);
        cands.push_back({300, q});
    }
    if (p->costmodel || default_costmodel()) {
        sptrsv_transform_params_t q = *prm;
        q.select_mode = SPTRSV_SELECT_COSTMODEL;
        q.solve_mode = SPTRSV_SOLVE_SYNCFREE;
        q.lanes_per_row = 1;
        CKS(sptrsv_transform(p, &q, stream));
        const int code = p->chosen_depth;
        if (code >= 0 && code < kThinOnly)
            add(code, SPTRSV_SELECT_FIXED, code, 0, 0, 0);
        else if (code >= kThinOnly)
            add(code, SPTRSV_SELECT_HEURISTIC, 0, kThinRows, code - kThinOnly, kThinBudget);
    }
    DevArr<double> b, x;
    CK(b.alloc(std::max<int32_t>(p->n, 1)));
    CK(x.alloc(std::max<int32_t>(p->n, 1)));
    std::vector<double> ones(std::max<int32_t>(p->n, 1), 1.0);
    CK(cudaMemcpyAsync(b.p, ones.data(), ones.size() * sizeof(double), cudaMemcpyHostToDevice,
                       s));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double best_ms = 1e30;
    int best = 0;
    sptrsv_status_t st = SPTRSV_OK;
    // each candidate timed in one layout, 2 lanes per row on 128-thread
    // CTAs: the best or within a few per cent of the best of the staged
    // kernel on every plan measured; the winner is then tuned in full
    for (size_t i = 0; i < cands.size() && st == SPTRSV_OK; ++i) {
        for (int L : {2}) {
            sptrsv_transform_params_t q = cands[i].q;
            q.solve_mode = SPTRSV_SOLVE_SYNCFREE;
            q.lanes_per_row = L;
            q.block_threads = 128;
            q.grid_blocks = 0;
            q.tail_rows = -1;
            if ((st = sptrsv_transform(p, &q, stream)) != SPTRSV_OK) break;
            double ms = 1e30;
            for (int r = 0; r < 4 && st == SPTRSV_OK; ++r) {
                if (cudaEventRecord(e0, s) != cudaSuccess) st = SPTRSV_ERR_CUDA;
                if (st == SPTRSV_OK) st = solve_impl(p, b.p, x.p, 1, s);
                if (st == SPTRSV_OK && (cudaEventRecord(e1, s) != cudaSuccess ||
                                        cudaEventSynchronize(e1) != cudaSuccess))
                    st = SPTRSV_ERR_CUDA;
                float t = 0;
                if (st == SPTRSV_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
                    st = SPTRSV_ERR_CUDA;
                if (r > 0) ms = std::min(ms, (double)t);   // the first is the warm-up
            }
            if (st == SPTRSV_OK) st = sync_status(p, s);
            if (st == SPTRSV_OK && ms < best_ms) {
                best_ms = ms;
                best = (int)i;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SPTRSV_OK) return st;
    CKS(sptrsv_transform(p, &cands[best].q, stream));
    p->chosen_depth = cands[best].code;
    p->prm.select_mode = SPTRSV_SELECT_AUTO;
    p->transform_ms = now_ms() - t0;
    return SPTRSV_OK;
}

}  // namespace

extern "C" {

const char *sptrsv_status_string(sptrsv_status_t s) {
    switch (s) {
    case SPTRSV_OK: return "ok";
    case SPTRSV_ERR_INVALID_ARG: return "invalid argument";
    case SPTRSV_ERR_NOT_LOWER: return "matrix is not lower triangular (or column out of range)";
    case SPTRSV_ERR_UNSORTED: return "CSR row pointers or columns are not sorted";
    case SPTRSV_ERR_ZERO_DIAG: return "zero on the diagonal";
    case SPTRSV_ERR_MISSING_DIAG: return "diagonal entry missing";
    case SPTRSV_ERR_OOM: return "device out of memory";
    case SPTRSV_ERR_CUDA: return "CUDA runtime error";
    case SPTRSV_ERR_TIMEOUT: return "a bounded device wait timed out";
    case SPTRSV_ERR_BAD_STATE: return "plan in a bad state (call order or earlier failure)";
    case SPTRSV_ERR_UNSUPPORTED: return "unsupported size or mode";
    case SPTRSV_ERR_BREAKDOWN: return "iteration breakdown (non-finite residual or curvature <= 0)";
    case SPTRSV_ERR_CODEGEN: return "generated code: runtime compiler missing or source rejected";
    }
    return "unknown status";
}

void sptrsv_default_params(sptrsv_transform_params_t *prm) {
    if (!prm) return;
    std::memset(prm, 0, sizeof(*prm));
    prm->select_mode = SPTRSV_SELECT_HEURISTIC;
    prm->depth = 2;
    prm->thin_rows = 0;
    prm->max_depth = 8;
    prm->flop_budget = 0.10;
    prm->max_row_fill = 1024;
    prm->solve_mode = SPTRSV_SOLVE_AUTO;
    prm->precision = SPTRSV_F64;
    prm->ir_tol = 1e-15;
    prm->ir_max_iter = 8;
    prm->lanes_per_row = 0;
    prm->block_threads = 0;
    prm->cta_run_rows = 0;
    prm->wait_timeout_ms = 5000;
    prm->grid_blocks = 0;
    prm->poll_backoff_ns = -1;
    prm->nrhs_hint = 1;
}

sptrsv_status_t sptrsv_analyze(int32_t n, int64_t nnz, const int32_t *d_row_ptr,
                               const int32_t *d_col, const double *d_val,
                               sptrsv_stream_t stream, sptrsv_plan_t *out) {
    return sptrsv_analyze_ex(n, nnz, d_row_ptr, d_col, d_val, SPTRSV_OP_LOWER, stream, out);
}

sptrsv_status_t sptrsv_analyze_ex(int32_t n, int64_t nnz, const int32_t *d_row_ptr,
                                  const int32_t *d_col, const double *d_val, int32_t op,
                                  sptrsv_stream_t stream, sptrsv_plan_t *out) {
    if (!out) return SPTRSV_ERR_INVALID_ARG;
    if (op < SPTRSV_OP_LOWER || op > SPTRSV_OP_UPPER_TRANS) return SPTRSV_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 0 || nnz < 0 || nnz > INT32_MAX) return SPTRSV_ERR_INVALID_ARG;
    if (n > 0 && (!d_row_ptr || (nnz > 0 && (!d_col || !d_val)))) return SPTRSV_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const double t0 = now_ms();
    sptrsv_plan_s *p = new sptrsv_plan_s();
    auto fail = [&](sptrsv_status_t st) {
        delete p;
        return st;
    };
    auto cuda_fail = [&](cudaError_t e) {
        (void)cudaGetLastError();
        delete p;
        return cuda_status(e);
    };
#define CKP(x)                                                                 \
    do {                                                                       \
        cudaError_t _e = (x);                                                  \
        if (_e != cudaSuccess) return cuda_fail(_e);                           \
    } while (0)
    CKP(cudaGetDevice(&p->device));
    CKP(cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device));
    CKP(cudaDeviceGetAttribute(&p->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor,
                               p->device));
    p->n = n;
    p->nnz = nnz;
    p->op = op;
    sptrsv_default_params(&p->prm);
    p->prm.select_mode = SPTRSV_SELECT_NONE;
    p->prm.solve_mode = SPTRSV_SOLVE_BARRIER;
    resolve_params(p, &p->prm);
    CKP(p->status.alloc(1));
    CKP(cudaMemsetAsync(p->status.p, 0, sizeof(DevStatus), s));
    CKP(p->lnorm.alloc(1));
    CKP(cudaMemsetAsync(p->lnorm.p, 0, sizeof(unsigned long long), s));
    CKP(p->row_ptr.alloc((size_t)n + 1));
    CKP(p->col.alloc(nnz));
    CKP(p->val.alloc(nnz));
    if (n == 0) {
        p->nlev = 0;
        p->h_level_ptr.assign(1, 0);
        CKP(p->level_ptr.alloc(1));
        CKP(cudaMemsetAsync(p->level_ptr.p, 0, sizeof(int32_t), s));
        CKP(cudaStreamSynchronize(s));
        p->analyze_ms = now_ms() - t0;
        *out = p;
        return SPTRSV_OK;
    }
    CKP(cudaMemcpyAsync(p->row_ptr.p, d_row_ptr, ((size_t)n + 1) * sizeof(int32_t),
                        cudaMemcpyDeviceToDevice, s));
    if (nnz > 0) {
        CKP(cudaMemcpyAsync(p->col.p, d_col, nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        CKP(cudaMemcpyAsync(p->val.p, d_val, nnz * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    DevArr<unsigned long long> err;
    CKP(err.alloc(1));
    // other operators: bring op(A) to lower-triangular form (csrc/operator.cu)
    if (op != SPTRSV_OP_LOWER) {
        CKP(cudaMemsetAsync(err.p, 0xff, sizeof(unsigned long long), s));
        CKP(launch_csr_check(n, nnz, p->row_ptr.p, p->col.p, err.p, s));
        unsigned long long h_chk = 0;
        CKP(cudaMemcpyAsync(&h_chk, err.p, sizeof(h_chk), cudaMemcpyDeviceToHost, s));
        CKP(cudaStreamSynchronize(s));
        if (h_chk != ~0ull) return fail((sptrsv_status_t)(h_chk & 0xff));
        auto replace = [&](DevArr<int32_t> &rp, DevArr<int32_t> &cl, DevArr<double> &vl) {
            p->row_ptr = std::move(rp);
            p->col = std::move(cl);
            p->val = std::move(vl);
        };
        if (op == SPTRSV_OP_LOWER_TRANS || op == SPTRSV_OP_UPPER_TRANS) {
            DevArr<int32_t> trp, tcl, rows, order, cnt;
            DevArr<double> tvl;
            DevArr<int64_t> stmp0;
            DevArr<char> rtmp;
            CKP(trp.alloc((size_t)n + 1));
            CKP(tcl.alloc(nnz));
            CKP(tvl.alloc(nnz));
            CKP(rows.alloc(nnz));
            CKP(order.alloc(nnz));
            CKP(cnt.alloc(n));
            CKP(stmp0.alloc(scan_tmp_elems(n)));
            CKP(rtmp.alloc(radix_tmp_bytes((int32_t)nnz)));
            CKP(launch_csr_transpose(n, nnz, p->row_ptr.p, p->col.p, p->val.p, trp.p, tcl.p,
                                     tvl.p, rows.p, order.p, cnt.p, stmp0.p, rtmp.p, s));
            CKP(cudaStreamSynchronize(s));
            replace(trp, tcl, tvl);
        }
        if (op == SPTRSV_OP_UPPER || op == SPTRSV_OP_LOWER_TRANS) {
            DevArr<int32_t> rrp, rcl;
            DevArr<double> rvl;
            CKP(rrp.alloc((size_t)n + 1));
            CKP(rcl.alloc(nnz));
            CKP(rvl.alloc(nnz));
            CKP(launch_csr_reverse(n, nnz, p->row_ptr.p, p->col.p, p->val.p, rrp.p, rcl.p,
                                   rvl.p, s));
            CKP(cudaStreamSynchronize(s));
            replace(rrp, rcl, rvl);
            p->rev = true;
        }
    }
    // validation
    CKP(cudaMemsetAsync(err.p, 0xff, sizeof(unsigned long long), s));
    CKP(p->offdeg.alloc(n));
    CKP(launch_validate(n, nnz, p->row_ptr.p, p->col.p, p->val.p, p->offdeg.p, err.p,
                        p->lnorm.p, s));
    unsigned long long h_err = 0;
    CKP(cudaMemcpyAsync(&h_err, err.p, sizeof(h_err), cudaMemcpyDeviceToHost, s));
    CKP(cudaStreamSynchronize(s));
    if (h_err != ~0ull) return fail((sptrsv_status_t)(h_err & 0xff));
    {
        DevArr<unsigned long long> bins;
        CKP(bins.alloc(4));
        CKP(cudaMemsetAsync(bins.p, 0, 4 * sizeof(unsigned long long), s));
        CKP(launch_offdeg_hist(n, p->offdeg.p, bins.p, s));
        unsigned long long hb[4];
        CKP(cudaMemcpyAsync(hb, bins.p, sizeof(hb), cudaMemcpyDeviceToHost, s));
        CKP(cudaStreamSynchronize(s));
        for (int k = 0; k < 4; ++k) p->offdeg_hist[k] = (int64_t)hb[k];
    }
    // levels of DAG_L by a synchronisation-free pass in row order
    DevArr<int32_t> nlev_d;
    CKP(nlev_d.alloc(1));
    CKP(p->level.alloc(n));
    CKP(launch_levels_syncfree(n, p->row_ptr.p, p->col.p, p->level.p, nlev_d.p, p->status.p,
                               timeout_ns(p), p->num_sms, s));
    int32_t nlev = 0;
    CKP(cudaMemcpyAsync(&nlev, nlev_d.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    {
        sptrsv_status_t st = sync_status(p, s);
        if (st != SPTRSV_OK) return fail(st);
    }
    if (nlev <= 0) return fail(SPTRSV_ERR_BAD_STATE);
    p->nlev = nlev;
    // rows ordered by (level, row), then the first position of every level
    CKP(p->perm.alloc(n));
    CKP(p->level_ptr.alloc((size_t)nlev + 1));
    {
        DevArr<char> rtmp;
        CKP(rtmp.alloc(radix_tmp_bytes(n)));
        CKP(launch_level_perm(n, p->level.p, nlev, p->perm.p, rtmp.p, s));
        CKP(launch_level_ptr(n, p->level.p, p->perm.p, nlev, p->level_ptr.p, s));
        CKP(cudaStreamSynchronize(s));
    }
    p->h_level_ptr.resize((size_t)nlev + 1);
    CKP(cudaMemcpy(p->h_level_ptr.data(), p->level_ptr.p, ((size_t)nlev + 1) * sizeof(int32_t),
                   cudaMemcpyDeviceToHost));
    if (p->h_level_ptr[nlev] != n) return fail(SPTRSV_ERR_BAD_STATE);
    // plain level-set structure
    {
        sptrsv_status_t st = choose_segments(p, s);
        if (st == SPTRSV_OK) {
            p->cfg = SolveConfig{};
            p->cfg.L = 1;
            p->cfg.block_threads = 512;
            p->cfg.grid = p->num_sms;
            p->cfg.cta_run_rows = 0;
            st = apply_config(p, s);
        }
        if (st == SPTRSV_OK) st = count_terms(p, s);
        if (st != SPTRSV_OK) return fail(st);
    }
#undef CKP
    p->analyze_ms = now_ms() - t0;
    *out = p;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_transform(sptrsv_plan_t p, const sptrsv_transform_params_t *prm,
                                 sptrsv_stream_t stream) {
    if (!p || !prm) return SPTRSV_ERR_INVALID_ARG;
    if (p->latched != SPTRSV_OK) return SPTRSV_ERR_BAD_STATE;
    if (prm->select_mode == SPTRSV_SELECT_AUTO) return select_auto(p, prm, stream);
    if (prm->select_mode < 0 || prm->select_mode > 6 || prm->solve_mode < 0 ||
        prm->solve_mode > 2 || (prm->precision != SPTRSV_F64 && prm->precision != SPTRSV_F32_IR))
        return SPTRSV_ERR_INVALID_ARG;
    if (prm->lanes_per_row != 0 && prm->lanes_per_row != 1 && prm->lanes_per_row != 2 &&
        prm->lanes_per_row != 4 && prm->lanes_per_row != 8 && prm->lanes_per_row != 16 &&
        prm->lanes_per_row != 32)
        return SPTRSV_ERR_INVALID_ARG;
    if (prm->block_threads != 0 &&
        (prm->block_threads < 64 || prm->block_threads > 512 || prm->block_threads % 32))
        return SPTRSV_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const double t0 = now_ms();
    resolve_params(p, prm);
    if (p->n == 0) {
        p->transform_ms = now_ms() - t0;
        return SPTRSV_OK;
    }
    p->s64 = SolveStruct<double>{};
    p->s32 = SolveStruct<float>{};
    CKS(choose_segments(p, s));
    CKS(build_rewritten(p, s));
    // provisional config: requested or default launch shape
    SolveConfig c;
    c.syncfree = p->prm.solve_mode == SPTRSV_SOLVE_SYNCFREE;
    c.block_threads = p->prm.block_threads > 0 ? p->prm.block_threads : 512;
    c.grid = p->prm.grid_blocks > 0 ? p->prm.grid_blocks
                                    : (c.syncfree ? 0 : p->num_sms);
    c.backoff_ns = p->prm.poll_backoff_ns > 0 ? p->prm.poll_backoff_ns : 0;
    c.L = 1;
    p->cfg = c;
    CKS(build_struct<double>(p, p->s64, 1, s));
    CKS(count_terms(p, s));
    c.L = p->prm.lanes_per_row > 0 ? p->prm.lanes_per_row : auto_lanes(p);
    if (p->prm.nrhs_hint > 1 && p->prm.lanes_per_row <= 0) {
        // several columns: one lane per (row, column), a chunk's rows in one pass
        c.L = 1;
        while (c.L < p->prm.nrhs_hint) c.L *= 2;
    }
    c.cta_run_rows = p->prm.cta_run_rows < 0 ? 0
                     : p->prm.cta_run_rows > 0 ? p->prm.cta_run_rows
                                               : c.block_threads / c.L;
    if (c.syncfree) c.cta_run_rows = 0;
    c.tail_rows = p->prm.tail_rows > 0 && (c.syncfree || c.cta_run_rows <= 0) ? p->prm.tail_rows
                                                                             : 0;
    p->cfg = c;
    CKS(apply_config(p, s));
    if (p->prm.solve_mode == SPTRSV_SOLVE_AUTO) CKS(autotune(p, s));
    CKS(sync_status(p, s));
    p->transform_ms = now_ms() - t0;
    return SPTRSV_OK;
}

void sptrsv_autotune_cache_clear(void) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache.clear();
}

sptrsv_status_t sptrsv_solve(sptrsv_plan_t p, const double *d_b, double *d_x, int32_t nrhs,
                             sptrsv_stream_t stream) {
    if (!p) return SPTRSV_ERR_INVALID_ARG;
    if (p->latched != SPTRSV_OK) return SPTRSV_ERR_BAD_STATE;
    if (nrhs < 1) return SPTRSV_ERR_INVALID_ARG;
    if (p->n == 0) return SPTRSV_OK;
    if (!d_b || !d_x) return SPTRSV_ERR_INVALID_ARG;
    const size_t bytes = (size_t)p->n * nrhs * sizeof(double);
    const char *b0 = (const char *)d_b, *x0 = (const char *)d_x;
    if (b0 < x0 + bytes && x0 < b0 + bytes) return SPTRSV_ERR_INVALID_ARG;
    return solve_impl(p, d_b, d_x, nrhs, (cudaStream_t)stream);
}

sptrsv_status_t sptrsv_check(sptrsv_plan_t p, sptrsv_stream_t stream) {
    if (!p) return SPTRSV_ERR_INVALID_ARG;
    if (p->latched != SPTRSV_OK) return p->latched;
    return sync_status(p, (cudaStream_t)stream);
}

sptrsv_status_t sptrsv_get_info(sptrsv_plan_t p, sptrsv_info_t *o) {
    if (!p || !o) return SPTRSV_ERR_INVALID_ARG;
    std::memset(o, 0, sizeof(*o));
    o->n = p->n;
    o->nnz = p->nnz;
    o->nlev = p->nlev;
    o->nlev_new = (int32_t)p->seg_first.size();
    o->rows_rewritten = p->rows_rewritten;
    o->nnz_x = p->nnz_x;
    o->nnz_b = p->nnz_b;
    o->flops_plain = plain_flops(p);
    o->flops_new = 2 * (p->nnz_x + p->nnz_b) + p->n;
    o->select_mode = p->prm.select_mode;
    o->solve_mode = p->cfg.syncfree ? SPTRSV_SOLVE_SYNCFREE : SPTRSV_SOLVE_BARRIER;
    o->precision = p->prm.precision;
    o->lanes_per_row = p->cfg.L;
    o->block_threads = p->cfg.block_threads;
    o->grid_blocks = p->n ? grid_for(p, 1, p->prm.precision == SPTRSV_F32_IR) : 0;
    o->cta_run_rows = p->cfg.cta_run_rows;
    o->thin_rows = p->thin_rows_used;
    o->max_depth = p->prm.max_depth;
    o->flop_budget = p->prm.flop_budget;
    o->num_sms = p->num_sms;
    o->poll_backoff_ns = p->cfg.backoff_ns;
    o->chosen_depth = p->chosen_depth;
    o->analyze_ms = p->analyze_ms;
    o->transform_ms = p->transform_ms;
    o->op = p->op;
    o->tuned_from_cache = p->tuned_from_cache ? 1 : 0;
    o->tail_rows = tail_active(p, 1) ? p->cfg.tail_rows : 0;
    o->tail_levels = tail_active(p, 1) ? p->tail.nlev : 0;
    o->codegen_segments = 0;
    if (tail_active(p, 1) && p->tail.gen_rows == p->prm.codegen_rows)
        for (const TailSeg &sg : p->tail.segs) o->codegen_segments += sg.gen.fn != nullptr;
    o->codegen_ms = p->tail.gen_ms;
    o->stage_z = p->prm.precision == SPTRSV_F32_IR ? 0 : stage_width(p, p->s64);
    if (p->status.p) {
        DevStatus h;
        if (cudaMemcpy(&h, p->status.p, sizeof(h), cudaMemcpyDeviceToHost) == cudaSuccess)
            o->ir_iters_last = h.ir_iters;
    }
    return SPTRSV_OK;
}

void sptrsv_plan_destroy(sptrsv_plan_t p) {
    if (!p) return;
    cudaDeviceSynchronize();
    delete p;
}

sptrsv_status_t sptrsv_get_levels(sptrsv_plan_t p, int32_t *d_level, int32_t *d_level_ptr,
                                  int32_t *d_perm, sptrsv_stream_t stream) {
    if (!p) return SPTRSV_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (p->n == 0) {
        if (d_level_ptr) CK(cudaMemsetAsync(d_level_ptr, 0, sizeof(int32_t), s));
        CK(cudaStreamSynchronize(s));
        return SPTRSV_OK;
    }
    if (d_level)
        CK(cudaMemcpyAsync(d_level, p->level.p, p->n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    if (d_level_ptr)
        CK(cudaMemcpyAsync(d_level_ptr, p->level_ptr.p, ((size_t)p->nlev + 1) * sizeof(int32_t),
                           cudaMemcpyDeviceToDevice, s));
    if (d_perm)
        CK(cudaMemcpyAsync(d_perm, p->perm.p, p->n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    if (p->rev) CK(launch_levels_reverse(p->n, d_level, d_perm, s));
    CK(cudaStreamSynchronize(s));
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_get_segments(sptrsv_plan_t p, int32_t *h_first, int32_t *h_depth) {
    if (!p) return SPTRSV_ERR_INVALID_ARG;
    for (size_t i = 0; i < p->seg_first.size(); ++i) {
        if (h_first) h_first[i] = p->seg_first[i];
        if (h_depth) h_depth[i] = p->seg_depth[i];
    }
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_get_transformed(sptrsv_plan_t p, int32_t *d_new_level, int64_t *d_xptr,
                                       int32_t *d_xcol, double *d_xval, int64_t *d_bptr,
                                       int32_t *d_bcol, double *d_bw, sptrsv_stream_t stream) {
    if (!p) return SPTRSV_ERR_INVALID_ARG;
    if (p->latched != SPTRSV_OK) return SPTRSV_ERR_BAD_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t n = p->n;
    if (n == 0) return SPTRSV_OK;
    if ((d_xcol || d_xval) && !d_xptr) return SPTRSV_ERR_INVALID_ARG;
    if ((d_bcol || d_bw) && !d_bptr) return SPTRSV_ERR_INVALID_ARG;
    DevArr<int64_t> xc, bc, tmp, xp, bp;
    CK(xc.alloc(n));
    CK(bc.alloc(n));
    CK(tmp.alloc(scan_tmp_elems(n)));
    CK(launch_export_count(p->s64.nchunks, p->s64.L, p->s64.meta.p, p->s64.ecol.p,
                           p->s64.row_id.p, p->n, xc.p, bc.p, s));
    int64_t *xptr = d_xptr, *bptr = d_bptr;
    if (!xptr) {
        CK(xp.alloc(n + 1));
        xptr = xp.p;
    }
    if (!bptr) {
        CK(bp.alloc(n + 1));
        bptr = bp.p;
    }
    CK(exclusive_scan_i64_i64(xc.p, xptr, n, tmp.p, s));
    CK(exclusive_scan_i64_i64(bc.p, bptr, n, tmp.p, s));
    CK(launch_export_fill(p->s64.nchunks, p->s64.L, p->s64.meta.p, p->s64.ecol.p, p->s64.eval.p,
                          p->s64.row_id.p, p->s64.chunk_level.p, p->s64.chunk_run_p0.p, p->n,
                          xptr, bptr, d_xcol, d_xval, d_bcol, d_bw, d_new_level, s));
    CK(cudaStreamSynchronize(s));
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_set_costmodel(sptrsv_plan_t p, sptrsv_mlp_t net) {
    if (!p) return SPTRSV_ERR_INVALID_ARG;
    p->costmodel = net;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_costmodel_features(sptrsv_plan_t p, const int32_t *h_depths, int32_t nd,
                                          float *h_feat, sptrsv_stream_t stream) {
    if (!p || nd < 0 || (nd > 0 && (!h_depths || !h_feat))) return SPTRSV_ERR_INVALID_ARG;
    if (p->latched != SPTRSV_OK) return SPTRSV_ERR_BAD_STATE;
    for (int32_t i = 0; i < nd; ++i) {
        const int32_t c = h_depths[i];
        if (c < 0 || (c > 16 && c < kThinOnly) || c > kThinOnly + 16)
            return SPTRSV_ERR_INVALID_ARG;
        CKS(candidate_features(p, h_depths[i], h_feat + (int64_t)i * kCostFeatures,
                               (cudaStream_t)stream));
    }
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_set_profiling(sptrsv_plan_t p, int32_t on) {
    if (!p) return SPTRSV_ERR_INVALID_ARG;
    if (on && !p->prof_ev[0]) {
        CK(cudaEventCreate(&p->prof_ev[0]));
        CK(cudaEventCreate(&p->prof_ev[1]));
    }
    p->profiling = on != 0;
    p->prof_valid = false;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_last_kernel_ms(sptrsv_plan_t p, float *ms) {
    if (!p || !ms) return SPTRSV_ERR_INVALID_ARG;
    if (!p->prof_valid) return SPTRSV_ERR_BAD_STATE;
    CK(cudaEventSynchronize(p->prof_ev[1]));
    CK(cudaEventElapsedTime(ms, p->prof_ev[0], p->prof_ev[1]));
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_level_features(sptrsv_plan_t p, int32_t lifts, float *h_feat,
                                      sptrsv_stream_t stream) {
    if (!p || lifts < 0 || lifts > 16 || (p->nlev > 0 && !h_feat)) return SPTRSV_ERR_INVALID_ARG;
    if (p->latched != SPTRSV_OK) return SPTRSV_ERR_BAD_STATE;
    const int32_t nlev = p->nlev;
    if (nlev == 0) return SPTRSV_OK;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<unsigned long long> acc((size_t)nlev * 11);
    {
        DevArr<unsigned long long> d;
        CK(d.alloc(acc.size()));
        CK(cudaMemsetAsync(d.p, 0, acc.size() * sizeof(unsigned long long), s));
        CK(launch_level_counts(p->n, p->row_ptr.p, p->col.p, p->level.p, d.p, s));
        CK(cudaMemcpyAsync(acc.data(), d.p, acc.size() * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    FillQuery fo{p, s, p->prm.max_row_fill, {}};
    std::vector<std::pair<int32_t, int32_t>> qs;
    for (int32_t l = 1; l < nlev; ++l)
        for (int32_t r = 1; r <= std::min(lifts, l); ++r) qs.emplace_back(l, r);
    CKS(fo.run(qs));
    const int F = 11 + lifts;
    for (int32_t l = 0; l < nlev; ++l) {
        float *f = h_feat + (size_t)l * F;
        for (int k = 0; k < 11; ++k) f[k] = (float)acc[(size_t)l * 11 + k];
        for (int r = 1; r <= lifts; ++r)
            f[10 + r] = r <= l ? (float)fo.cache[{l, r}] : 0.f;   // -1: over the fill cap
    }
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_segment_features(sptrsv_plan_t p, int32_t d_max, float *h_feat,
                                        uint8_t *h_ok, sptrsv_stream_t stream) {
    if (!p || !h_feat || !h_ok || d_max < 0 || d_max > 16) return SPTRSV_ERR_INVALID_ARG;
    if (p->latched != SPTRSV_OK) return SPTRSV_ERR_BAD_STATE;
    std::vector<float> feat;
    std::vector<uint8_t> ok;
    CKS(segment_table(p, d_max, (cudaStream_t)stream, feat, ok));
    std::memcpy(h_feat, feat.data(), feat.size() * sizeof(float));
    std::memcpy(h_ok, ok.data(), ok.size());
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_level_times(sptrsv_plan_t p, const double *d_b, double *d_x,
                                   int32_t reps, double *h_us, sptrsv_stream_t stream) {
    if (!p || !d_b || !d_x || !h_us || reps < 1) return SPTRSV_ERR_INVALID_ARG;
    if (p->latched != SPTRSV_OK) return SPTRSV_ERR_BAD_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t nl = p->s64.nlev;
    const int stz = stage_width(p, p->s64);
    if (p->prm.precision == SPTRSV_F32_IR || !p->cfg.syncfree || stz <= 0 ||
        tail_active(p, 1) || !p->s64.built || nl <= 0)
        return SPTRSV_ERR_UNSUPPORTED;
    SolveData<double> sd = p->s64.view();
    sd.backoff_ns = p->cfg.backoff_ns;
    sd.stage_z = stz;
    if (!p->cfg.sched_lm) sd.sched = nullptr;
    DevArr<unsigned long long> ns;
    CK(ns.alloc((size_t)nl + 1));
    sd.level_ns = ns.p;
    LaunchCfg lc{p->cfg.block_threads, grid_for(p, 1, false)};
    if (lc.grid <= 0) return SPTRSV_ERR_CUDA;
    std::vector<std::vector<double>> inc(nl);
    std::vector<unsigned long long> h((size_t)nl + 1);
    for (int32_t r = 0; r < reps; ++r) {
        CK(cudaMemsetAsync(ns.p, 0, ((size_t)nl + 1) * sizeof(unsigned long long), s));
        CK(launch_solve<double>(sd, d_b, d_x, p->n, 1, 1, true, lc, p->status.p, timeout_ns(p),
                                false, s));
        CK(cudaMemcpyAsync(h.data(), ns.p, h.size() * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, s));
        CKS(sync_status(p, s));
        unsigned long long prev = h[0];
        for (int32_t g = 0; g < nl; ++g) {
            const unsigned long long t = std::max(prev, h[1 + g]);
            inc[g].push_back((double)(t - prev) * 1e-3);
            prev = t;
        }
    }
    for (int32_t g = 0; g < nl; ++g) {
        std::sort(inc[g].begin(), inc[g].end());
        h_us[g] = inc[g][inc[g].size() / 2];
    }
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_codegen_source(sptrsv_plan_t p, int32_t seg, char *buf, size_t cap,
                                      size_t *len) {
    if (!p || !len || seg < 0) return SPTRSV_ERR_INVALID_ARG;
    if (p->latched != SPTRSV_OK) return SPTRSV_ERR_BAD_STATE;
    if (!p->tail.built || (size_t)seg >= p->tail.segs.size()) return SPTRSV_ERR_INVALID_ARG;
    const TailSeg &sg = p->tail.segs[seg];
    if (!sg.gen.fn || p->tail.gen_rows != p->prm.codegen_rows) return SPTRSV_ERR_BAD_STATE;
    std::string src;
    bool thin = false;
    CKS(codegen_source(sg, src, thin));
    if (!thin) return SPTRSV_ERR_BAD_STATE;
    *len = src.size();
    if (buf && cap > 0) {
        const size_t k = std::min(cap - 1, src.size());
        std::memcpy(buf, src.data(), k);
        buf[k] = 0;
    }
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_critical_path(sptrsv_plan_t p, int32_t hop_weight, int64_t *h_cp,
                                     sptrsv_stream_t stream) {
    if (!p || !h_cp) return SPTRSV_ERR_INVALID_ARG;
    if (p->latched != SPTRSV_OK) return SPTRSV_ERR_BAD_STATE;
    *h_cp = 0;
    if (p->n == 0) return SPTRSV_OK;
    const SolveStruct<double> &ss = p->s64;
    if (!ss.built) return SPTRSV_ERR_BAD_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t hop = hop_weight > 0 ? hop_weight : 16;
    DevArr<int64_t> fin;
    CK(fin.alloc(p->n));
    CK(cudaMemsetAsync(fin.p, 0, (size_t)p->n * sizeof(int64_t), s));
    const int32_t *p0 = ss.run_encoded > 0 ? ss.chunk_run_p0.p : nullptr;
    for (int32_t l = 0; l < ss.nlev; ++l)
        CK(launch_critpath_level(ss.h_lvl_chunk[l], ss.h_lvl_chunk[l + 1], ss.L, p->n,
                                 ss.meta.p, ss.ecol.p, ss.row_id.p, p0, hop, fin.p, s));
    std::vector<int64_t> h(p->n);
    CK(cudaMemcpyAsync(h.data(), fin.p, h.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *h_cp = *std::max_element(h.begin(), h.end());
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_debug_inject_wait(sptrsv_plan_t p, int32_t row) {
    if (!p || row < 0 || row >= p->n) return SPTRSV_ERR_INVALID_ARG;
    if (p->latched != SPTRSV_OK) return SPTRSV_ERR_BAD_STATE;
    // find the row's solve position and chunk on the host, then rewrite its
    // first slot (a padded slot is added if the row has none) to read x[row]
    std::vector<int32_t> row_id(p->n);
    CK(cudaMemcpy(row_id.data(), p->s64.row_id.p, p->n * sizeof(int32_t), cudaMemcpyDeviceToHost));
    int32_t pos = -1;
    for (int32_t i = 0; i < p->n; ++i)
        if (row_id[i] == row) { pos = i; break; }
    if (pos < 0) return SPTRSV_ERR_BAD_STATE;
    std::vector<int4> meta(p->s64.nchunks);
    CK(cudaMemcpy(meta.data(), p->s64.meta.p, meta.size() * sizeof(int4), cudaMemcpyDeviceToHost));
    for (int32_t c = 0; c < p->s64.nchunks; ++c) {
        const int4 m = meta[c];
        if (pos < m.x || pos >= m.x + m.y) continue;
        if (m.z == 0) return SPTRSV_ERR_UNSUPPORTED;  // row without any slot
        const int32_t k = pos - m.x;
        const int64_t slot = (int64_t)m.w + (int64_t)k * p->s64.L;
        CK(cudaMemcpy(p->s64.ecol.p + slot, &row, sizeof(int32_t), cudaMemcpyHostToDevice));
        if (p->s32.built)
            CK(cudaMemcpy(p->s32.ecol.p + slot, &row, sizeof(int32_t), cudaMemcpyHostToDevice));
        // the single-CTA tail's records were built from the old entries: drop
        // them and keep the tail off for good (a later transform would build
        // it from the injected entries, and the tail kernel does not wait), so
        // that the main kernel, whose waits are bounded, solves every level
        p->tail = TailStruct{};
        p->injected = true;
        // the staged kernels read the chunks' blobs: rebuild them
        const bool had64 = p->s64.blob_valid, had32 = p->s32.blob_valid;
        p->s64.blob_valid = p->s32.blob_valid = false;
        if (had64) CKS(build_blob(p->s64, 0));
        if (had32) CKS(build_blob(p->s32, 0));
        return SPTRSV_OK;
    }
    return SPTRSV_ERR_BAD_STATE;
}

}  // extern "C"
