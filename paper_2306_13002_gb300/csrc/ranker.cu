// Learned cost model for rewriter variants: a 3-layer FP32 MLP, trained and evaluated by
// hand-written kernels.
//
// The paper extracts with a fixed analytical cost (Sec. V-B) and notes that better costs
// are future work. Here a small multilayer perceptron learns the measured run time of
// variants from their static features, and `acs_variant_rank` orders variants by its
// prediction (or by the analytical cost when no model is given).
//
// Model: x (F features, standardised with the training set's mean and deviation) ->
// h1 = relu(W1 x + b1) (H) -> h2 = relu(W2 h1 + b2) (H) -> y = w3 . h2 + b3, the
// standardised log of the run time. Loss: weighted mean squared error over the training set,
// sample weight w_i = exp(-a t_i) / mean_j exp(-a t_j) of its standardised log time t_i (a = 0:
// plain MSE; a > 0 weighs the fast variants, which decide the pick, more).
// Optimiser: Adam (Kingma & Ba, 2015; beta1 0.9, beta2 0.999, eps 1e-8), full batch.
// Parameter buffer (floats): mu[F] sd[F] tmu tsd W1[H*F] b1[H] W2[H*H] b2[H] w3[H] b3.
// Per epoch three kernels: forward (a block per sample, a thread per hidden unit),
// per-sample backward (the same shape), and gradient + Adam (a thread per parameter that
// sums its gradient over the samples in a fixed order, so training is deterministic).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <numeric>
#include <string>
#include <vector>

#include "acs_internal.cuh"

namespace acs {
namespace {

struct Layout {
    int F, H;
    size_t mu, sd, tmu, tsd, W1, b1, W2, b2, w3, b3, P;
    __host__ __device__ Layout(int f, int h) : F(f), H(h) {
        mu = 0;
        sd = mu + F;
        tmu = sd + F;
        tsd = tmu + 1;
        W1 = tsd + 1;
        b1 = W1 + (size_t)H * F;
        W2 = b1 + H;
        b2 = W2 + (size_t)H * H;
        w3 = b2 + H;
        b3 = w3 + H;
        P = b3 + 1;
    }
};

// Forward pass; also keeps the activations when H1/H2 are non-null (training).
__global__ void mlp_forward(const float* __restrict__ X, const float* __restrict__ prm, int F, int H, float* H1,
                            float* H2, float* Y, int standardise) {
    extern __shared__ float sh[];
    float* x = sh;            // F
    float* h1 = sh + F;       // H
    float* h2 = h1 + H;       // H
    const int s = blockIdx.x, j = threadIdx.x;
    const Layout L(F, H);
    for (int f = j; f < F; f += blockDim.x) {
        const float v = X[(size_t)s * F + f];
        x[f] = standardise ? (v - prm[L.mu + f]) / prm[L.sd + f] : v;
    }
    __syncthreads();
    if (j < H) {
        float a = prm[L.b1 + j];
        for (int f = 0; f < F; ++f) a += prm[L.W1 + (size_t)j * F + f] * x[f];
        a = a > 0.f ? a : 0.f;
        h1[j] = a;
        if (H1) H1[(size_t)s * H + j] = a;
    }
    __syncthreads();
    if (j < H) {
        float a = prm[L.b2 + j];
        for (int k = 0; k < H; ++k) a += prm[L.W2 + (size_t)j * H + k] * h1[k];
        a = a > 0.f ? a : 0.f;
        h2[j] = a;
        if (H2) H2[(size_t)s * H + j] = a;
    }
    __syncthreads();
    if (j == 0) {
        float y = prm[L.b3];
        for (int k = 0; k < H; ++k) y += prm[L.w3 + k] * h2[k];
        Y[s] = y;
    }
}

__global__ void mlp_backward_sample(const float* __restrict__ T, const float* __restrict__ Wt, const float* __restrict__ prm,
                                    int F, int H, int n, const float* __restrict__ H1, const float* __restrict__ H2,
                                    const float* __restrict__ Y, float* DH1, float* DH2, float* DY) {
    extern __shared__ float sh[];
    float* dh2 = sh;
    const int s = blockIdx.x, j = threadIdx.x;
    const Layout L(F, H);
    const float dy = 2.f * Wt[s] * (Y[s] - T[s]) / (float)n;
    if (j == 0) DY[s] = dy;
    if (j < H) {
        const float g = H2[(size_t)s * H + j] > 0.f ? dy * prm[L.w3 + j] : 0.f;
        dh2[j] = g;
        DH2[(size_t)s * H + j] = g;
    }
    __syncthreads();
    if (j < H) {
        float a = 0.f;
        for (int k = 0; k < H; ++k) a += prm[L.W2 + (size_t)k * H + j] * dh2[k];
        DH1[(size_t)s * H + j] = H1[(size_t)s * H + j] > 0.f ? a : 0.f;
    }
}

// Gradient of the loss with respect to parameter p (a thread per parameter, samples summed in
// order), then either the Adam update of p (grad == NULL) or the gradient stored in grad[p].
__global__ void mlp_grad_adam(const float* __restrict__ X, const float* __restrict__ H1, const float* __restrict__ H2,
                              const float* __restrict__ DH1, const float* __restrict__ DH2, const float* __restrict__ DY,
                              float* prm, float* m, float* v, int F, int H, int n, int step, float lr, float* grad) {
    const Layout L(F, H);
    const size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (p >= L.P) return;
    if (p < L.W1) {  // mu, sd, tmu, tsd are fixed
        if (grad) grad[p] = 0.f;
        return;
    }
    float g = 0.f;
    if (p < L.b1) {
        const int j = (int)((p - L.W1) / F), f = (int)((p - L.W1) % F);
        for (int s = 0; s < n; ++s) {
            const float xf = (X[(size_t)s * F + f] - prm[L.mu + f]) / prm[L.sd + f];
            g += DH1[(size_t)s * H + j] * xf;
        }
    } else if (p < L.W2) {
        const int j = (int)(p - L.b1);
        for (int s = 0; s < n; ++s) g += DH1[(size_t)s * H + j];
    } else if (p < L.b2) {
        const int j = (int)((p - L.W2) / H), k = (int)((p - L.W2) % H);
        for (int s = 0; s < n; ++s) g += DH2[(size_t)s * H + j] * H1[(size_t)s * H + k];
    } else if (p < L.w3) {
        const int j = (int)(p - L.b2);
        for (int s = 0; s < n; ++s) g += DH2[(size_t)s * H + j];
    } else if (p < L.b3) {
        const int k = (int)(p - L.w3);
        for (int s = 0; s < n; ++s) g += DY[s] * H2[(size_t)s * H + k];
    } else {
        for (int s = 0; s < n; ++s) g += DY[s];
    }
    if (grad) {
        grad[p] = g;
        return;
    }
    const float b1 = 0.9f, b2 = 0.999f;
    const float mm = b1 * m[p] + (1.f - b1) * g;
    const float vv = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float mh = mm / (1.f - powf(b1, (float)step));
    const float vh = vv / (1.f - powf(b2, (float)step));
    prm[p] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

__global__ void copy_column(const float* __restrict__ X, int F, int col, int n, float* out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) out[s] = X[(size_t)s * F + col];
}

struct Ws {
    float *H1, *H2, *Y, *DH1, *DH2, *DY, *T, *W, *m, *v;
};
size_t ws_floats(int n, int H, size_t P) { return 4 * (size_t)n * H + 4 * (size_t)n + 2 * P; }
Ws carve(float* base, int n, int H, size_t P) {
    Ws w;
    w.H1 = base;
    w.H2 = w.H1 + (size_t)n * H;
    w.DH1 = w.H2 + (size_t)n * H;
    w.DH2 = w.DH1 + (size_t)n * H;
    w.Y = w.DH2 + (size_t)n * H;
    w.DY = w.Y + n;
    w.T = w.DY + n;
    w.W = w.T + n;
    w.m = w.W + n;
    w.v = w.m + P;
    return w;
}

// Sample weights of the loss: exp(-a t_i) normalised to mean 1 (t: standardised log times).
std::vector<float> loss_weights(const std::vector<float>& tstd, float a) {
    std::vector<double> w(tstd.size());
    double sum = 0.0;
    for (size_t i = 0; i < w.size(); ++i) sum += (w[i] = std::exp(-(double)a * tstd[i]));
    std::vector<float> out(w.size());
    for (size_t i = 0; i < w.size(); ++i) out[i] = (float)(w[i] * (double)w.size() / sum);
    return out;
}

}  // namespace

size_t ranker_param_count(int F, int H) { return F < 1 || H < 1 ? 0 : Layout(F, H).P; }
size_t ranker_ws_bytes(int n, int F, int H) {
    return n < 1 || F < 1 || H < 1 ? 0 : sizeof(float) * ws_floats(n, H, Layout(F, H).P);
}

acs_status ranker_train(const float* feats, const float* times, int n, int F, int H, int epochs, float lr,
                        float fast_weight, unsigned long long seed, float* params, void* ws, size_t ws_bytes,
                        cudaStream_t s) {
    const Layout L(F, H);
    if (ws_bytes < ranker_ws_bytes(n, F, H)) return fail(ACS_ERR_WORKSPACE, "ranker workspace too small");
    // Standardisation statistics and the initial weights are computed on the host.
    std::vector<float> hx((size_t)n * F), ht(n);
    if (cudaMemcpyAsync(hx.data(), feats, hx.size() * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(ht.data(), times, ht.size() * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return launch_status("ranker_train: copying the training set");
    std::vector<float> p(L.P, 0.f), tlog(n);
    for (int f = 0; f < F; ++f) {
        double mu = 0, var = 0;
        for (int i = 0; i < n; ++i) mu += hx[(size_t)i * F + f];
        mu /= n;
        for (int i = 0; i < n; ++i) var += (hx[(size_t)i * F + f] - mu) * (hx[(size_t)i * F + f] - mu);
        const double sd = std::sqrt(var / n);
        p[L.mu + f] = (float)mu;
        p[L.sd + f] = (float)(sd > 1e-6 ? sd : 1.0);
    }
    for (int i = 0; i < n; ++i) {
        if (!(ht[i] > 0.f)) return fail(ACS_ERR_INVALID, "training time %d is not positive", i);
        tlog[i] = std::log(ht[i]);
    }
    double tm = 0, tv = 0;
    for (float t : tlog) tm += t;
    tm /= n;
    for (float t : tlog) tv += (t - tm) * (t - tm);
    const double tsd = std::sqrt(tv / n);
    p[L.tmu] = (float)tm;
    p[L.tsd] = (float)(tsd > 1e-6 ? tsd : 1.0);
    std::vector<float> tstd(n);
    for (int i = 0; i < n; ++i) tstd[i] = (float)((tlog[i] - tm) / p[L.tsd]);
    uint64_t ctr = 0;
    auto uni = [&]() {
        uint64_t z = seed + (++ctr) * 0x9E3779B97F4A7C15ULL;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    const double a1 = std::sqrt(6.0 / F), a2 = std::sqrt(6.0 / H);
    for (size_t q = 0; q < (size_t)H * F; ++q) p[L.W1 + q] = (float)((2 * uni() - 1) * a1);
    for (size_t q = 0; q < (size_t)H * H; ++q) p[L.W2 + q] = (float)((2 * uni() - 1) * a2);
    for (int q = 0; q < H; ++q) p[L.w3 + q] = (float)((2 * uni() - 1) * a2);
    Ws w = carve(static_cast<float*>(ws), n, H, L.P);
    const std::vector<float> wts = loss_weights(tstd, fast_weight);
    if (cudaMemcpyAsync(params, p.data(), L.P * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(w.T, tstd.data(), n * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(w.W, wts.data(), n * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(w.m, 0, 2 * L.P * 4, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return launch_status("ranker_train: uploading the initial model");
    const int tb = H < 32 ? 32 : ((H + 31) / 32) * 32;
    const size_t sh_f = sizeof(float) * (F + 2 * H), sh_b = sizeof(float) * H;
    const unsigned pg = (unsigned)((L.P + 255) / 256);
    for (int e = 1; e <= epochs; ++e) {   // epochs == 0: the initial model only
        mlp_forward<<<n, tb, sh_f, s>>>(feats, params, F, H, w.H1, w.H2, w.Y, 1);
        mlp_backward_sample<<<n, tb, sh_b, s>>>(w.T, w.W, params, F, H, n, w.H1, w.H2, w.Y, w.DH1, w.DH2, w.DY);
        mlp_grad_adam<<<pg, 256, 0, s>>>(feats, w.H1, w.H2, w.DH1, w.DH2, w.DY, params, w.m, w.v, F, H, n, e, lr,
                                         nullptr);
    }
    return launch_status("ranker training kernels");
}

acs_status ranker_gradient(const float* feats, const float* times, int n, int F, int H, const float* params,
                           float fast_weight, float* grad, void* ws, size_t ws_bytes, cudaStream_t s) {
    const Layout L(F, H);
    if (ws_bytes < ranker_ws_bytes(n, F, H)) return fail(ACS_ERR_WORKSPACE, "ranker workspace too small");
    // The target: the standardised log time, with the statistics stored in the model.
    std::vector<float> ht(n), st(2);
    if (cudaMemcpyAsync(ht.data(), times, n * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(st.data(), params + L.tmu, 2 * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return launch_status("ranker_gradient: reading times and target scale");
    if (!(st[1] > 0.f)) return fail(ACS_ERR_NOMODEL, "model has no target scale");
    std::vector<float> tstd(n);
    for (int i = 0; i < n; ++i) {
        if (!(ht[i] > 0.f)) return fail(ACS_ERR_INVALID, "time %d is not positive", i);
        tstd[i] = (float)((std::log(ht[i]) - st[0]) / st[1]);
    }
    Ws w = carve(static_cast<float*>(ws), n, H, L.P);
    const std::vector<float> wts = loss_weights(tstd, fast_weight);
    if (cudaMemcpyAsync(w.T, tstd.data(), n * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(w.W, wts.data(), n * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return launch_status("ranker_gradient: uploading targets");
    const int tb = H < 32 ? 32 : ((H + 31) / 32) * 32;
    float* prm = const_cast<float*>(params);   // read only when grad is set
    mlp_forward<<<n, tb, sizeof(float) * (F + 2 * H), s>>>(feats, params, F, H, w.H1, w.H2, w.Y, 1);
    mlp_backward_sample<<<n, tb, sizeof(float) * H, s>>>(w.T, w.W, params, F, H, n, w.H1, w.H2, w.Y, w.DH1, w.DH2,
                                                          w.DY);
    mlp_grad_adam<<<(unsigned)((L.P + 255) / 256), 256, 0, s>>>(feats, w.H1, w.H2, w.DH1, w.DH2, w.DY, prm, w.m, w.v,
                                                                 F, H, n, 1, 0.f, grad);
    if (cudaStreamSynchronize(s) != cudaSuccess) return launch_status("ranker_gradient kernels");
    return launch_status("ranker_gradient kernels");
}

// Model file: "acs-ranker-model 1", then "F H P", then the P parameters one per line in
// hexadecimal floating point (%a), so that a load gives back the same bits.
acs_status ranker_save(const char* path, const float* params, int F, int H) {
    const Layout L(F, H);
    std::vector<float> p(L.P);
    // The model may have been trained on any stream (non-blocking ones do not order with this
    // copy): wait for all work on the device first.
    if (cudaDeviceSynchronize() != cudaSuccess) return launch_status("ranker_save: waiting for the device");
    if (cudaMemcpy(p.data(), params, L.P * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return launch_status("ranker_save: reading the model");
    FILE* f = fopen(path, "w");
    if (!f) return fail(ACS_ERR_INVALID, "cannot open %s for writing", path);
    bool ok = fprintf(f, "acs-ranker-model 1\n%d %d %zu\n", F, H, L.P) > 0;
    for (size_t q = 0; q < L.P && ok; ++q) ok = fprintf(f, "%a\n", (double)p[q]) > 0;
    ok = (fclose(f) == 0) && ok;
    return ok ? ACS_OK : fail(ACS_ERR_INVALID, "writing %s failed", path);
}

acs_status ranker_load(const char* path, float* params, size_t capacity, int* F_out, int* H_out) {
    FILE* f = fopen(path, "r");
    if (!f) return fail(ACS_ERR_INVALID, "cannot open %s", path);
    int ver = 0, F = 0, H = 0;
    size_t P = 0;
    char magic[32] = {0};
    if (fscanf(f, "%31s %d", magic, &ver) != 2 || std::string(magic) != "acs-ranker-model" || ver != 1 ||
        fscanf(f, "%d %d %zu", &F, &H, &P) != 3 || F < 1 || F > 1024 || H < 1 || H > 1024 ||
        P != Layout(F, H).P) {
        fclose(f);
        return fail(ACS_ERR_INVALID, "%s is not an acs-ranker-model 1 file", path);
    }
    std::vector<float> p(P);
    for (size_t q = 0; q < P; ++q) {
        double v;
        if (fscanf(f, "%la", &v) != 1 || !std::isfinite(v)) {
            fclose(f);
            return fail(ACS_ERR_INVALID, "%s: parameter %zu is missing or not finite", path, q);
        }
        p[q] = (float)v;
    }
    fclose(f);
    if (F_out) *F_out = F;
    if (H_out) *H_out = H;
    if (!params) return ACS_OK;   // size query
    if (capacity < P) return fail(ACS_ERR_WORKSPACE, "model needs %zu floats, buffer holds %zu", P, capacity);
    // Kernels still reading an earlier model from `params` may run on any stream.
    if (cudaDeviceSynchronize() != cudaSuccess) return launch_status("ranker_load: waiting for the device");
    if (cudaMemcpy(params, p.data(), P * 4, cudaMemcpyHostToDevice) != cudaSuccess)
        return launch_status("ranker_load: uploading the model");
    return ACS_OK;
}

acs_status ranker_predict(const float* feats, int n, int F, int H, const float* params, float* scores, cudaStream_t s) {
    const int tb = H < 32 ? 32 : ((H + 31) / 32) * 32;
    mlp_forward<<<n, tb, sizeof(float) * (F + 2 * H), s>>>(feats, params, F, H, nullptr, nullptr, scores, 1);
    return launch_status("mlp_forward");
}

acs_status analytical_scores(const float* feats, int n, int F, float* scores, cudaStream_t s) {
    copy_column<<<(n + 255) / 256, 256, 0, s>>>(feats, F, 0, n, scores);
    return launch_status("copy_column");
}

acs_status ranker_denormalise(const float* params, int F, int H, std::vector<float>& y) {
    const Layout L(F, H);
    float st[2];
    if (cudaMemcpy(st, params + L.tmu, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess)
        return launch_status("reading the target scale");
    for (auto& v : y) v = std::exp(v * st[1] + st[0]);
    return ACS_OK;
}

}  // namespace acs
