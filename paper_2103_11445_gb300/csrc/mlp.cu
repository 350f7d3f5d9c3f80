// Cost-model network: 3-layer perceptron (F -> H -> H -> 1, ReLU, FP32) that
// predicts the log solve time of a rewrite choice.  The paper leaves the row
// choice to the programmer (Sec. IV); this network makes it from measured
// timings.  Forward, backward (MSE loss) and Adam are hand-written kernels;
// every reduction runs in a fixed order (deterministic).
//
// Parameter layout (one flat FP32 array): W1[F][H], b1[H], W2[H][H], b2[H],
// W3[H][1], b3[1]; row-major, X is [N][F].
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "plan.cuh"

using namespace sptrsv;

struct sptrsv_mlp_s {
    int32_t F = 0, H = 0;
    int64_t nparams = 0;
    DevArr<float> params, grads, m, v;
    DevArr<float> z1, z2, y, dy, dz1, dz2, loss;  // activations for the last batch size
    int64_t cap = 0;                               // samples the activation buffers hold
    int64_t step = 0;
    float feat_mean[64] = {}, feat_std[64] = {};  // input normalisation (host copy)
    bool has_norm = false;
};

namespace {

struct Off {
    int64_t W1, b1, W2, b2, W3, b3, total;
};
Off offsets(int F, int H) {
    Off o;
    o.W1 = 0;
    o.b1 = o.W1 + (int64_t)F * H;
    o.W2 = o.b1 + H;
    o.b2 = o.W2 + (int64_t)H * H;
    o.W3 = o.b2 + H;
    o.b3 = o.W3 + H;
    o.total = o.b3 + 1;
    return o;
}

// z[i][h] = sum_f a[i][f] W[f][h] + b[h]; r = relu(z) stored over z when relu
__global__ void dense_kernel(const float *__restrict__ a, const float *__restrict__ W,
                             const float *__restrict__ b, float *__restrict__ z, int N, int K,
                             int H) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * H) return;
    const int i = (int)(t / H), h = (int)(t % H);
    float s = b[h];
    for (int k = 0; k < K; ++k) s = fmaf(a[(int64_t)i * K + k], W[(int64_t)k * H + h], s);
    z[t] = s;
}

__global__ void relu_copy_kernel(const float *__restrict__ z, float *__restrict__ r, int64_t n) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) r[t] = z[t] > 0.f ? z[t] : 0.f;
}

// dy = 2 (y - target) / N and loss = mean (y - target)^2 (one block, fixed order)
__global__ void loss_kernel(const float *__restrict__ y, const float *__restrict__ tgt,
                            float *__restrict__ dy, float *__restrict__ loss, int N) {
    __shared__ float part[256];
    float s = 0.f;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const float e = y[i] - tgt[i];
        dy[i] = 2.f * e / (float)N;
        s = fmaf(e, e, s);
    }
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot = 0.f;
        for (int k = 0; k < (int)blockDim.x; ++k) tot += part[k];
        *loss = tot / (float)N;
    }
}

// gW[k][h] = sum_i a[i][k] g[i][h] (a = layer input, g = gradient w.r.t. z);
// gb[h] = sum_i g[i][h].  One thread per weight, samples in order.
__global__ void weight_grad_kernel(const float *__restrict__ a, const float *__restrict__ g,
                                   float *__restrict__ gW, float *__restrict__ gb, int N, int K,
                                   int H, int a_relu) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < K * H) {
        const int k = t / H, h = t % H;
        float s = 0.f;
        for (int i = 0; i < N; ++i) {
            float av = a[(int64_t)i * K + k];
            if (a_relu) av = av > 0.f ? av : 0.f;
            s = fmaf(av, g[(int64_t)i * H + h], s);
        }
        gW[t] = s;
    } else if (t < K * H + H) {
        const int h = t - K * H;
        float s = 0.f;
        for (int i = 0; i < N; ++i) s += g[(int64_t)i * H + h];
        gb[h] = s;
    }
}

// ga[i][k] = (sum_h g[i][h] W[k][h]) * (z[i][k] > 0)
__global__ void back_dense_kernel(const float *__restrict__ g, const float *__restrict__ W,
                                  const float *__restrict__ z, float *__restrict__ ga, int N,
                                  int K, int H) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * K) return;
    const int i = (int)(t / K), k = (int)(t % K);
    float s = 0.f;
    for (int h = 0; h < H; ++h) s = fmaf(g[(int64_t)i * H + h], W[(int64_t)k * H + h], s);
    ga[t] = z[t] > 0.f ? s : 0.f;
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float gt = g[t];
    const float mt = b1 * m[t] + (1.f - b1) * gt;
    const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
    m[t] = mt;
    v[t] = vt;
    p[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
}

unsigned blocks(int64_t n, int bs = 256) { return (unsigned)((n + bs - 1) / bs); }

// Column statistics of X [N][F]: one block per feature, FP64 sums in a fixed
// order (per-thread strided partial sums, then thread 0 adds them in order).
__global__ void column_stats_kernel(const float *__restrict__ X, int N, int F,
                                    double *__restrict__ mean, double *__restrict__ var) {
    __shared__ double ps[256], pq[256];
    const int f = blockIdx.x;
    double s = 0.0, q = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double v = X[(int64_t)i * F + f];
        s += v;
        q = fma(v, v, q);
    }
    ps[threadIdx.x] = s;
    pq[threadIdx.x] = q;
    __syncthreads();
    if (threadIdx.x == 0) {
        double ts = 0.0, tq = 0.0;
        for (int k = 0; k < (int)blockDim.x; ++k) {
            ts += ps[k];
            tq += pq[k];
        }
        const double m = ts / N;
        mean[f] = m;
        var[f] = fmax(tq / N - m * m, 0.0);
    }
}

__global__ void normalize_kernel(const float *__restrict__ X, float *__restrict__ Xn, int64_t n,
                                 int F, const float *__restrict__ mean,
                                 const float *__restrict__ inv_std) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int f = (int)(t % F);
    Xn[t] = (X[t] - mean[f]) * inv_std[f];
}

sptrsv_status_t ensure_cap(sptrsv_mlp_t net, int64_t N) {
    if (N <= net->cap) return SPTRSV_OK;
    const int64_t H = net->H;
    if (net->z1.alloc(N * H) || net->z2.alloc(N * H) || net->y.alloc(N) || net->dy.alloc(N) ||
        net->dz1.alloc(N * H) || net->dz2.alloc(N * H))
        return SPTRSV_ERR_OOM;
    net->cap = N;
    return SPTRSV_OK;
}

// forward pass into net->z1 / z2 (pre-activations) and y
cudaError_t forward(sptrsv_mlp_t net, const float *X, int N, cudaStream_t s) {
    const Off o = offsets(net->F, net->H);
    const float *P = net->params.p;
    const int F = net->F, H = net->H;
    dense_kernel<<<blocks((int64_t)N * H), 256, 0, s>>>(X, P + o.W1, P + o.b1, net->z1.p, N, F, H);
    // layer 2 reads relu(z1): materialise it in dz1 (scratch) for the dense kernel
    relu_copy_kernel<<<blocks((int64_t)N * H), 256, 0, s>>>(net->z1.p, net->dz1.p, (int64_t)N * H);
    dense_kernel<<<blocks((int64_t)N * H), 256, 0, s>>>(net->dz1.p, P + o.W2, P + o.b2, net->z2.p,
                                                       N, H, H);
    relu_copy_kernel<<<blocks((int64_t)N * H), 256, 0, s>>>(net->z2.p, net->dz2.p, (int64_t)N * H);
    dense_kernel<<<blocks(N), 256, 0, s>>>(net->dz2.p, P + o.W3, P + o.b3, net->y.p, N, H, 1);
    return cudaGetLastError();
}

// gradients of mean (y - t)^2 into net->grads (after forward)
cudaError_t backward(sptrsv_mlp_t net, const float *X, const float *tgt, int N, cudaStream_t s) {
    const Off o = offsets(net->F, net->H);
    const float *P = net->params.p;
    float *G = net->grads.p;
    const int F = net->F, H = net->H;
    loss_kernel<<<1, 256, 0, s>>>(net->y.p, tgt, net->dy.p, net->loss.p, N);
    // layer 3: input relu(z2)
    weight_grad_kernel<<<blocks((int64_t)H + 1), 256, 0, s>>>(net->z2.p, net->dy.p, G + o.W3,
                                                              G + o.b3, N, H, 1, 1);
    back_dense_kernel<<<blocks((int64_t)N * H), 256, 0, s>>>(net->dy.p, P + o.W3, net->z2.p,
                                                            net->dz2.p, N, H, 1);
    // layer 2: input relu(z1)
    weight_grad_kernel<<<blocks((int64_t)H * H + H), 256, 0, s>>>(net->z1.p, net->dz2.p, G + o.W2,
                                                                  G + o.b2, N, H, H, 1);
    back_dense_kernel<<<blocks((int64_t)N * H), 256, 0, s>>>(net->dz2.p, P + o.W2, net->z1.p,
                                                            net->dz1.p, N, H, H);
    // layer 1: input X
    weight_grad_kernel<<<blocks((int64_t)F * H + H), 256, 0, s>>>(X, net->dz1.p, G + o.W1,
                                                                  G + o.b1, N, F, H, 0);
    return cudaGetLastError();
}

}  // namespace

namespace sptrsv {
// Normalises h_feat [count][F] with the network's stored statistics and
// returns the predictions in h_pred (synchronises the stream).
// Predictions of the network for `count` raw feature rows (host): the rows
// are standardised on the device by the same kernel the training uses
// (sptrsv_mlp_normalize), so that a selection sees exactly the network's
// training-time arithmetic.
sptrsv_status_t costmodel_predict(sptrsv_mlp_t net, const float *h_feat, int count,
                                  float *h_pred, cudaStream_t s) {
    if (!net || count <= 0) return SPTRSV_ERR_INVALID_ARG;
    const int F = net->F;
    DevArr<float> dx;
    if (dx.alloc((size_t)count * F)) return SPTRSV_ERR_OOM;
    if (cudaMemcpyAsync(dx.p, h_feat, (size_t)count * F * sizeof(float), cudaMemcpyHostToDevice,
                        s))
        return SPTRSV_ERR_CUDA;
    const sptrsv_status_t st = sptrsv_mlp_normalize(net, dx.p, count, dx.p, s);
    if (st != SPTRSV_OK) return st;
    if (ensure_cap(net, count) != SPTRSV_OK) return SPTRSV_ERR_OOM;
    if (forward(net, dx.p, count, s) != cudaSuccess) return SPTRSV_ERR_CUDA;
    if (cudaMemcpyAsync(h_pred, net->y.p, count * sizeof(float), cudaMemcpyDeviceToHost, s) ||
        cudaStreamSynchronize(s))
        return SPTRSV_ERR_CUDA;
    return SPTRSV_OK;
}
// The process-wide default networks of SELECT_COSTMODEL
// (sptrsv_costmodel_load) and SELECT_SEGMODEL (sptrsv_segmodel_load); a
// network loaded from a file is owned by the library, one handed over by
// set_default stays the caller's.
std::mutex g_default_mu;
sptrsv_mlp_t g_default_net = nullptr;
bool g_default_owned = false;
sptrsv_mlp_t g_segment_net = nullptr;
bool g_segment_owned = false;
sptrsv_mlp_t default_costmodel() {
    std::lock_guard<std::mutex> lock(g_default_mu);
    return g_default_net;
}
sptrsv_mlp_t default_segmodel() {
    std::lock_guard<std::mutex> lock(g_default_mu);
    return g_segment_net;
}
// Replaces a default network; returns the old one if the library owned it.
sptrsv_mlp_t swap_default(sptrsv_mlp_t &slot, bool &owned, sptrsv_mlp_t net, bool own) {
    std::lock_guard<std::mutex> lock(g_default_mu);
    sptrsv_mlp_t old = owned && slot != net ? slot : nullptr;
    slot = net;
    owned = net && own;
    return old;
}
}  // namespace sptrsv

namespace {
// Network file (little-endian): 8 bytes "SPTRSVNN", int32 version (1), F, H,
// has_norm; float32 params[nparams(F, H)], mean[F], std[F].
constexpr char kNetMagic[8] = {'S', 'P', 'T', 'R', 'S', 'V', 'N', 'N'};
constexpr int32_t kNetVersion = 1;
}  // namespace

extern "C" {

SPTRSV_API sptrsv_status_t sptrsv_mlp_create(int32_t n_in, int32_t hidden, const float *h_params,
                                             sptrsv_mlp_t *out) {
    if (!out || n_in < 1 || n_in > 64 || hidden < 1 || hidden > 1024 || !h_params)
        return SPTRSV_ERR_INVALID_ARG;
    *out = nullptr;
    sptrsv_mlp_s *net = new sptrsv_mlp_s();
    net->F = n_in;
    net->H = hidden;
    net->nparams = offsets(n_in, hidden).total;
    const size_t bytes = net->nparams * sizeof(float);
    if (net->params.alloc(net->nparams) || net->grads.alloc(net->nparams) ||
        net->m.alloc(net->nparams) || net->v.alloc(net->nparams) || net->loss.alloc(1)) {
        delete net;
        return SPTRSV_ERR_OOM;
    }
    if (cudaMemcpy(net->params.p, h_params, bytes, cudaMemcpyHostToDevice) ||
        cudaMemset(net->m.p, 0, bytes) || cudaMemset(net->v.p, 0, bytes) ||
        cudaMemset(net->grads.p, 0, bytes)) {
        (void)cudaGetLastError();
        delete net;
        return SPTRSV_ERR_CUDA;
    }
    *out = net;
    return SPTRSV_OK;
}

SPTRSV_API int64_t sptrsv_mlp_num_params(int32_t n_in, int32_t hidden) {
    return offsets(n_in, hidden).total;
}

SPTRSV_API sptrsv_status_t sptrsv_mlp_get_params(sptrsv_mlp_t net, float *h_params) {
    if (!net || !h_params) return SPTRSV_ERR_INVALID_ARG;
    if (cudaMemcpy(h_params, net->params.p, net->nparams * sizeof(float), cudaMemcpyDeviceToHost))
        return SPTRSV_ERR_CUDA;
    return SPTRSV_OK;
}

SPTRSV_API sptrsv_status_t sptrsv_mlp_set_normalization(sptrsv_mlp_t net, const float *h_mean,
                                                        const float *h_std) {
    if (!net || !h_mean || !h_std) return SPTRSV_ERR_INVALID_ARG;
    for (int f = 0; f < net->F; ++f) {
        net->feat_mean[f] = h_mean[f];
        net->feat_std[f] = h_std[f] > 0.f ? h_std[f] : 1.f;
    }
    net->has_norm = true;
    return SPTRSV_OK;
}

SPTRSV_API sptrsv_status_t sptrsv_mlp_forward(sptrsv_mlp_t net, const float *d_X, int32_t N,
                                              float *d_y, sptrsv_stream_t stream) {
    if (!net || N < 0 || (N > 0 && (!d_X || !d_y))) return SPTRSV_ERR_INVALID_ARG;
    if (N == 0) return SPTRSV_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (ensure_cap(net, N) != SPTRSV_OK) return SPTRSV_ERR_OOM;
    if (forward(net, d_X, N, s) != cudaSuccess) return SPTRSV_ERR_CUDA;
    if (cudaMemcpyAsync(d_y, net->y.p, N * sizeof(float), cudaMemcpyDeviceToDevice, s))
        return SPTRSV_ERR_CUDA;
    return SPTRSV_OK;
}

SPTRSV_API sptrsv_status_t sptrsv_mlp_grads(sptrsv_mlp_t net, const float *d_X,
                                            const float *d_target, int32_t N, float *d_grads,
                                            float *d_loss, sptrsv_stream_t stream) {
    if (!net || N < 1 || !d_X || !d_target) return SPTRSV_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (ensure_cap(net, N) != SPTRSV_OK) return SPTRSV_ERR_OOM;
    if (forward(net, d_X, N, s) || backward(net, d_X, d_target, N, s)) return SPTRSV_ERR_CUDA;
    if (d_grads && cudaMemcpyAsync(d_grads, net->grads.p, net->nparams * sizeof(float),
                                   cudaMemcpyDeviceToDevice, s))
        return SPTRSV_ERR_CUDA;
    if (d_loss && cudaMemcpyAsync(d_loss, net->loss.p, sizeof(float), cudaMemcpyDeviceToDevice, s))
        return SPTRSV_ERR_CUDA;
    return SPTRSV_OK;
}

SPTRSV_API sptrsv_status_t sptrsv_mlp_train_step(sptrsv_mlp_t net, const float *d_X,
                                                 const float *d_target, int32_t N, float lr,
                                                 float *d_loss, sptrsv_stream_t stream) {
    sptrsv_status_t st = sptrsv_mlp_grads(net, d_X, d_target, N, nullptr, d_loss, stream);
    if (st != SPTRSV_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    net->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)net->step), c2 = 1.f - powf(b2, (float)net->step);
    adam_kernel<<<blocks(net->nparams), 256, 0, s>>>(net->params.p, net->grads.p, net->m.p,
                                                     net->v.p, net->nparams, lr, b1, b2, 1e-8f,
                                                     c1, c2);
    return cudaGetLastError() == cudaSuccess ? SPTRSV_OK : SPTRSV_ERR_CUDA;
}

SPTRSV_API void sptrsv_mlp_destroy(sptrsv_mlp_t net) {
    if (!net) return;
    {
        std::lock_guard<std::mutex> lock(sptrsv::g_default_mu);
        if (sptrsv::g_default_net == net) {
            sptrsv::g_default_net = nullptr;
            sptrsv::g_default_owned = false;
        }
        if (sptrsv::g_segment_net == net) {
            sptrsv::g_segment_net = nullptr;
            sptrsv::g_segment_owned = false;
        }
    }
    cudaDeviceSynchronize();
    delete net;
}

SPTRSV_API sptrsv_status_t sptrsv_mlp_fit_normalization(sptrsv_mlp_t net, const float *d_X,
                                                        int32_t N, sptrsv_stream_t stream) {
    if (!net || N < 1 || !d_X) return SPTRSV_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int F = net->F;
    DevArr<double> mv;
    if (mv.alloc(2 * (size_t)F)) return SPTRSV_ERR_OOM;
    column_stats_kernel<<<F, 256, 0, s>>>(d_X, N, F, mv.p, mv.p + F);
    std::vector<double> h(2 * (size_t)F);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(h.data(), mv.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s) ||
        cudaStreamSynchronize(s))
        return SPTRSV_ERR_CUDA;
    for (int f = 0; f < F; ++f) {
        const double sd = std::sqrt(h[F + f]);
        net->feat_mean[f] = (float)h[f];
        net->feat_std[f] = sd > 1e-6 ? (float)sd : 1.f;
    }
    net->has_norm = true;
    return SPTRSV_OK;
}

SPTRSV_API sptrsv_status_t sptrsv_mlp_get_normalization(sptrsv_mlp_t net, float *h_mean,
                                                        float *h_std) {
    if (!net || !h_mean || !h_std) return SPTRSV_ERR_INVALID_ARG;
    for (int f = 0; f < net->F; ++f) {
        h_mean[f] = net->has_norm ? net->feat_mean[f] : 0.f;
        h_std[f] = net->has_norm ? net->feat_std[f] : 1.f;
    }
    return SPTRSV_OK;
}

SPTRSV_API sptrsv_status_t sptrsv_mlp_normalize(sptrsv_mlp_t net, const float *d_X, int32_t N,
                                                float *d_Xn, sptrsv_stream_t stream) {
    if (!net || N < 0 || (N > 0 && (!d_X || !d_Xn))) return SPTRSV_ERR_INVALID_ARG;
    if (N == 0) return SPTRSV_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int F = net->F;
    std::vector<float> h(2 * (size_t)F);
    for (int f = 0; f < F; ++f) {
        h[f] = net->has_norm ? net->feat_mean[f] : 0.f;
        h[F + f] = net->has_norm ? 1.f / net->feat_std[f] : 1.f;
    }
    DevArr<float> st;
    if (st.alloc(h.size())) return SPTRSV_ERR_OOM;
    const int64_t n = (int64_t)N * F;
    if (cudaMemcpyAsync(st.p, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, s))
        return SPTRSV_ERR_CUDA;
    normalize_kernel<<<blocks(n), 256, 0, s>>>(d_X, d_Xn, n, F, st.p, st.p + F);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s)) return SPTRSV_ERR_CUDA;
    return SPTRSV_OK;
}

SPTRSV_API sptrsv_status_t sptrsv_mlp_save(sptrsv_mlp_t net, const char *path) {
    if (!net || !path) return SPTRSV_ERR_INVALID_ARG;
    std::vector<float> params(net->nparams);
    if (cudaMemcpy(params.data(), net->params.p, net->nparams * sizeof(float),
                   cudaMemcpyDeviceToHost))
        return SPTRSV_ERR_CUDA;
    FILE *f = std::fopen(path, "wb");
    if (!f) return SPTRSV_ERR_INVALID_ARG;
    const int32_t hdr[4] = {kNetVersion, net->F, net->H, net->has_norm ? 1 : 0};
    bool ok = std::fwrite(kNetMagic, 1, 8, f) == 8 && std::fwrite(hdr, 4, 4, f) == 4 &&
              std::fwrite(params.data(), 4, params.size(), f) == params.size() &&
              std::fwrite(net->feat_mean, 4, net->F, f) == (size_t)net->F &&
              std::fwrite(net->feat_std, 4, net->F, f) == (size_t)net->F;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? SPTRSV_OK : SPTRSV_ERR_INVALID_ARG;
}

SPTRSV_API sptrsv_status_t sptrsv_mlp_load(const char *path, sptrsv_mlp_t *out) {
    if (!path || !out) return SPTRSV_ERR_INVALID_ARG;
    *out = nullptr;
    FILE *f = std::fopen(path, "rb");
    if (!f) return SPTRSV_ERR_INVALID_ARG;
    char magic[8];
    int32_t hdr[4];
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kNetMagic, 8) == 0 &&
              std::fread(hdr, 4, 4, f) == 4 && hdr[0] == kNetVersion && hdr[1] >= 1 &&
              hdr[1] <= 64 && hdr[2] >= 1 && hdr[2] <= 1024;
    std::vector<float> params, mean, sd;
    if (ok) {
        params.resize(offsets(hdr[1], hdr[2]).total);
        mean.resize(hdr[1]);
        sd.resize(hdr[1]);
        ok = std::fread(params.data(), 4, params.size(), f) == params.size() &&
             std::fread(mean.data(), 4, mean.size(), f) == mean.size() &&
             std::fread(sd.data(), 4, sd.size(), f) == sd.size();
        char extra;
        ok = ok && std::fread(&extra, 1, 1, f) == 0;   // nothing after the weights
    }
    std::fclose(f);
    if (!ok) return SPTRSV_ERR_INVALID_ARG;
    sptrsv_mlp_t net = nullptr;
    sptrsv_status_t st = sptrsv_mlp_create(hdr[1], hdr[2], params.data(), &net);
    if (st != SPTRSV_OK) return st;
    if (hdr[3]) sptrsv_mlp_set_normalization(net, mean.data(), sd.data());
    *out = net;
    return SPTRSV_OK;
}

SPTRSV_API sptrsv_status_t sptrsv_costmodel_load(const char *path) {
    sptrsv_mlp_t net = nullptr;
    sptrsv_status_t st = sptrsv_mlp_load(path, &net);
    if (st != SPTRSV_OK) return st;
    sptrsv_mlp_t old =
        sptrsv::swap_default(sptrsv::g_default_net, sptrsv::g_default_owned, net, true);
    if (old) {
        cudaDeviceSynchronize();
        delete old;
    }
    return SPTRSV_OK;
}

SPTRSV_API sptrsv_status_t sptrsv_costmodel_save(const char *path) {
    std::lock_guard<std::mutex> lock(sptrsv::g_default_mu);
    if (!sptrsv::g_default_net) return SPTRSV_ERR_BAD_STATE;
    return sptrsv_mlp_save(sptrsv::g_default_net, path);
}

SPTRSV_API sptrsv_status_t sptrsv_costmodel_set_default(sptrsv_mlp_t net) {
    sptrsv_mlp_t old =
        sptrsv::swap_default(sptrsv::g_default_net, sptrsv::g_default_owned, net, false);
    if (old) {
        cudaDeviceSynchronize();
        delete old;
    }
    return SPTRSV_OK;
}

SPTRSV_API sptrsv_status_t sptrsv_segmodel_load(const char *path) {
    sptrsv_mlp_t net = nullptr;
    sptrsv_status_t st = sptrsv_mlp_load(path, &net);
    if (st != SPTRSV_OK) return st;
    if (net->F != sptrsv::kSegFeatures) {
        delete net;
        return SPTRSV_ERR_INVALID_ARG;
    }
    sptrsv_mlp_t old =
        sptrsv::swap_default(sptrsv::g_segment_net, sptrsv::g_segment_owned, net, true);
    if (old) {
        cudaDeviceSynchronize();
        delete old;
    }
    return SPTRSV_OK;
}

SPTRSV_API sptrsv_status_t sptrsv_segmodel_set_default(sptrsv_mlp_t net) {
    if (net && net->F != sptrsv::kSegFeatures) return SPTRSV_ERR_INVALID_ARG;
    sptrsv_mlp_t old =
        sptrsv::swap_default(sptrsv::g_segment_net, sptrsv::g_segment_owned, net, false);
    if (old) {
        cudaDeviceSynchronize();
        delete old;
    }
    return SPTRSV_OK;
}

}  // extern "C"
