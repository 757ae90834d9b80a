// Learned cost model: a multilayer perceptron (3 hidden layers x 128 ReLU, one
// linear output) that predicts, from a plan's features, the log of its
// measured over its analytic contraction time (the planner adds the analytic
// log time back when it ranks candidates).  The paper divides a FLOP count by the GPU's FLOP rate
// (Eq. classical_runtime, §V) and finds the estimate consistently high
// (§VIII); this model is trained on timings the planner itself generates and
// ranks candidate plans.  Forward, backward and Adam run in this file's own
// CUDA kernels (FP32); the host code only orchestrates them.
//
// Parameter layout (flat, device): W1 [F x 128], b1, W2 [128 x 128], b2,
// W3 [128 x 128], b3, W4 [128 x 1], b4; rows of X are samples, Y = X W + b.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "tqc_internal.h"

struct tqc_costmodel {
    int n_in = 0;
    int64_t n_params = 0;
    float *d_theta = nullptr, *d_grad = nullptr, *d_m = nullptr, *d_v = nullptr;
    // activations for the current batch capacity
    int cap = 0;
    float *d_X = nullptr, *d_t = nullptr, *d_A[4] = {nullptr, nullptr, nullptr, nullptr}, *d_D[4] = {nullptr, nullptr, nullptr, nullptr};
    float *d_y = nullptr, *d_dy = nullptr, *d_loss = nullptr;
    std::vector<float> mean, stdv;  // feature standardisation
    float t_mean = 0.f, t_std = 1.f;
    int64_t adam_step = 0;
};

namespace tqc {
namespace {

constexpr int H = 128;
constexpr int TILE = 16;

// C[M x N] = op(A) op(B) (+ bias) with an optional ReLU, or masked by
// (mask > 0).  op(A) = A [M x K] or A^T with A [K x M]; op(B) = B [K x N] or
// B^T with B [N x K].  accumulate: C += result.
__global__ void mlp_gemm(const float *A, const float *B, float *C, int M, int N, int K, int transA, int transB,
                         const float *bias, const float *mask, int relu, int accumulate) {
    __shared__ float As[TILE][TILE + 1], Bs[TILE][TILE + 1];
    const int tx = threadIdx.x % TILE, ty = threadIdx.x / TILE;
    const int row = blockIdx.y * TILE + ty, col = blockIdx.x * TILE + tx;
    float acc = 0.f;
    for (int k0 = 0; k0 < K; k0 += TILE) {
        const int ka = k0 + tx, kb = k0 + ty;
        const int ar = blockIdx.y * TILE + ty;
        As[ty][tx] = (ar < M && ka < K) ? (transA ? A[(size_t)ka * M + ar] : A[(size_t)ar * K + ka]) : 0.f;
        const int bc = blockIdx.x * TILE + tx;
        Bs[ty][tx] = (kb < K && bc < N) ? (transB ? B[(size_t)bc * K + kb] : B[(size_t)kb * N + bc]) : 0.f;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TILE; ++k) acc = fmaf(As[ty][k], Bs[k][tx], acc);
        __syncthreads();
    }
    if (row < M && col < N) {
        if (bias) acc += bias[col];
        if (relu) acc = fmaxf(acc, 0.f);
        if (mask && !(mask[(size_t)row * N + col] > 0.f)) acc = 0.f;
        float *c = C + (size_t)row * N + col;
        *c = accumulate ? *c + acc : acc;
    }
}

// db[n] = sum over rows of D [M x N]
__global__ void mlp_colsum(const float *D, float *db, int M, int N) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += D[(size_t)m * N + n];
    db[n] = s;
}

// dy = 2 (y - t) / B and loss = mean (y - t)^2 (single block)
__global__ void mlp_mse(const float *y, const float *t, float *dy, float *loss, int B) {
    __shared__ float red[256];
    float s = 0.f;
    for (int i = threadIdx.x; i < B; i += blockDim.x) {
        const float d = y[i] - t[i];
        dy[i] = 2.f * d / (float)B;
        s += d * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0] / (float)B;
}

// Adam (Kingma & Ba): bias-corrected first and second moments
__global__ void mlp_adam(float *theta, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                         float eps, float c1, float c2) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void mlp_gather(const float *X, const float *t, const int *idx, float *Xb, float *tb, int B, int F) {
    const int i = blockIdx.x;
    if (i >= B) return;
    const int src = idx[i];
    for (int f = threadIdx.x; f < F; f += blockDim.x) Xb[(size_t)i * F + f] = X[(size_t)src * F + f];
    if (threadIdx.x == 0 && t) tb[i] = t[src];
}

void gemm(const float *A, const float *B, float *C, int M, int N, int K, int tA, int tB, const float *bias,
          const float *mask, int relu, int acc, cudaStream_t s) {
    dim3 grid((N + TILE - 1) / TILE, (M + TILE - 1) / TILE);
    mlp_gemm<<<grid, TILE * TILE, 0, s>>>(A, B, C, M, N, K, tA, tB, bias, mask, relu, acc);
}

struct Offs {
    int64_t w[4], b[4];
};
Offs offsets(int F) {
    Offs o;
    const int ins[4] = {F, H, H, H}, outs[4] = {H, H, H, 1};
    int64_t off = 0;
    for (int l = 0; l < 4; ++l) {
        o.w[l] = off;
        off += (int64_t)ins[l] * outs[l];
        o.b[l] = off;
        off += outs[l];
    }
    return o;
}

int64_t count_params(int F) { return (int64_t)F * H + H + 2 * ((int64_t)H * H + H) + H + 1; }

tqc_status ensure_cap(tqc_costmodel *cm, int B) {
    if (B <= cm->cap) return TQC_OK;
    cudaFree(cm->d_X);
    cudaFree(cm->d_t);
    cudaFree(cm->d_y);
    cudaFree(cm->d_dy);
    for (int l = 0; l < 4; ++l) {
        cudaFree(cm->d_A[l]);
        cudaFree(cm->d_D[l]);
    }
    cm->cap = 0;
    bool ok = cudaMalloc(&cm->d_X, sizeof(float) * (size_t)B * cm->n_in) == cudaSuccess &&
              cudaMalloc(&cm->d_t, sizeof(float) * B) == cudaSuccess &&
              cudaMalloc(&cm->d_y, sizeof(float) * B) == cudaSuccess &&
              cudaMalloc(&cm->d_dy, sizeof(float) * B) == cudaSuccess;
    for (int l = 0; l < 4 && ok; ++l)
        ok = cudaMalloc(&cm->d_A[l], sizeof(float) * (size_t)B * H) == cudaSuccess &&
             cudaMalloc(&cm->d_D[l], sizeof(float) * (size_t)B * H) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return fail(TQC_ERR_OOM, "cost-model activation buffers");
    }
    cm->cap = B;
    return TQC_OK;
}

// forward of the batch already in d_X (B rows); prediction in d_y
void forward(tqc_costmodel *cm, int B, cudaStream_t s) {
    const Offs o = offsets(cm->n_in);
    const float *th = cm->d_theta;
    gemm(cm->d_X, th + o.w[0], cm->d_A[0], B, H, cm->n_in, 0, 0, th + o.b[0], nullptr, 1, 0, s);
    gemm(cm->d_A[0], th + o.w[1], cm->d_A[1], B, H, H, 0, 0, th + o.b[1], nullptr, 1, 0, s);
    gemm(cm->d_A[1], th + o.w[2], cm->d_A[2], B, H, H, 0, 0, th + o.b[2], nullptr, 1, 0, s);
    gemm(cm->d_A[2], th + o.w[3], cm->d_y, B, 1, H, 0, 0, th + o.b[3], nullptr, 0, 0, s);
}

// loss and gradient (into d_grad) of the batch in d_X / d_t
void backward(tqc_costmodel *cm, int B, cudaStream_t s) {
    const Offs o = offsets(cm->n_in);
    const float *th = cm->d_theta;
    float *g = cm->d_grad;
    mlp_mse<<<1, 256, 0, s>>>(cm->d_y, cm->d_t, cm->d_dy, cm->d_loss, B);
    // layer 4: y = A3 W4 + b4
    gemm(cm->d_A[2], cm->d_dy, g + o.w[3], H, 1, B, 1, 0, nullptr, nullptr, 0, 0, s);
    mlp_colsum<<<1, 32, 0, s>>>(cm->d_dy, g + o.b[3], B, 1);
    // dZ3 = dy W4^T masked by A3 > 0
    gemm(cm->d_dy, th + o.w[3], cm->d_D[2], B, H, 1, 0, 1, nullptr, cm->d_A[2], 0, 0, s);
    for (int l = 2; l >= 1; --l) {
        gemm(cm->d_A[l - 1], cm->d_D[l], g + o.w[l], H, H, B, 1, 0, nullptr, nullptr, 0, 0, s);
        mlp_colsum<<<(H + 127) / 128, 128, 0, s>>>(cm->d_D[l], g + o.b[l], B, H);
        gemm(cm->d_D[l], th + o.w[l], cm->d_D[l - 1], B, H, H, 0, 1, nullptr, cm->d_A[l - 1], 0, 0, s);
    }
    gemm(cm->d_X, cm->d_D[0], g + o.w[0], cm->n_in, H, B, 1, 0, nullptr, nullptr, 0, 0, s);
    mlp_colsum<<<(H + 127) / 128, 128, 0, s>>>(cm->d_D[0], g + o.b[0], B, H);
}

uint64_t splitmix(uint64_t &x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double uniform01(uint64_t &x) { return (double)(splitmix(x) >> 11) * (1.0 / 9007199254740992.0); }

std::mutex g_load_mu;
std::map<std::string, tqc_costmodel *> g_loaded;  // learned planner: one model per path

}  // namespace

tqc_status costmodel_predict_host(tqc_costmodel *cm, const float *h_X, int n, float *h_y);

}  // namespace tqc

using namespace tqc;

#define CM_CUDA(call, what)                                                                  \
    do {                                                                                     \
        cudaError_t _e = (call);                                                             \
        if (_e != cudaSuccess) return fail(TQC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(_e)); \
    } while (0)

extern "C" {

tqc_status tqc_costmodel_create(int32_t n_features, uint64_t seed, tqc_costmodel_t *out) {
    if (!out || n_features < 1 || n_features > 4096) return fail(TQC_ERR_INVALID, "bad cost-model arguments");
    *out = nullptr;
    tqc_costmodel *cm = new tqc_costmodel;
    cm->n_in = n_features;
    cm->n_params = count_params(n_features);
    size_t bytes = sizeof(float) * (size_t)cm->n_params;
    if (cudaMalloc(&cm->d_theta, bytes) != cudaSuccess || cudaMalloc(&cm->d_grad, bytes) != cudaSuccess ||
        cudaMalloc(&cm->d_m, bytes) != cudaSuccess || cudaMalloc(&cm->d_v, bytes) != cudaSuccess ||
        cudaMalloc(&cm->d_loss, sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        tqc_costmodel_destroy(cm);
        return fail(TQC_ERR_OOM, "cost-model parameters");
    }
    // He-uniform weights, zero biases, from a seeded counter-based generator
    std::vector<float> h(cm->n_params, 0.f);
    const Offs o = offsets(n_features);
    const int ins[4] = {n_features, H, H, H}, outs[4] = {H, H, H, 1};
    uint64_t st = seed;
    for (int l = 0; l < 4; ++l) {
        const double lim = std::sqrt(6.0 / ins[l]);
        for (int64_t i = 0; i < (int64_t)ins[l] * outs[l]; ++i) h[o.w[l] + i] = (float)((2 * uniform01(st) - 1) * lim);
    }
    cudaMemcpy(cm->d_theta, h.data(), bytes, cudaMemcpyHostToDevice);
    cudaMemset(cm->d_m, 0, bytes);
    cudaMemset(cm->d_v, 0, bytes);
    cm->mean.assign(n_features, 0.f);
    cm->stdv.assign(n_features, 1.f);
    *out = cm;
    return TQC_OK;
}

tqc_status tqc_costmodel_destroy(tqc_costmodel_t cm) {
    if (!cm) return fail(TQC_ERR_INVALID, "NULL cost model");
    cudaFree(cm->d_theta);
    cudaFree(cm->d_grad);
    cudaFree(cm->d_m);
    cudaFree(cm->d_v);
    cudaFree(cm->d_loss);
    cudaFree(cm->d_X);
    cudaFree(cm->d_t);
    cudaFree(cm->d_y);
    cudaFree(cm->d_dy);
    for (int l = 0; l < 4; ++l) {
        cudaFree(cm->d_A[l]);
        cudaFree(cm->d_D[l]);
    }
    delete cm;
    return TQC_OK;
}

tqc_status tqc_costmodel_params(tqc_costmodel_t cm, float *h_out, int32_t *n) {
    if (!cm || !n) return fail(TQC_ERR_INVALID, "NULL argument");
    if (h_out) {
        if (*n < cm->n_params) return fail(TQC_ERR_INVALID, "parameter buffer too small");
        CM_CUDA(cudaMemcpy(h_out, cm->d_theta, sizeof(float) * cm->n_params, cudaMemcpyDeviceToHost), "params");
    }
    *n = (int32_t)cm->n_params;
    return TQC_OK;
}

tqc_status tqc_costmodel_set_params(tqc_costmodel_t cm, const float *h_in, int32_t n) {
    if (!cm || !h_in || n != cm->n_params) return fail(TQC_ERR_INVALID, "parameter count mismatch");
    CM_CUDA(cudaMemcpy(cm->d_theta, h_in, sizeof(float) * n, cudaMemcpyHostToDevice), "set params");
    return TQC_OK;
}

tqc_status tqc_costmodel_grad(tqc_costmodel_t cm, const float *h_X, const float *h_t, int32_t n, float *h_grad,
                              float *h_loss) {
    if (!cm || !h_X || !h_t || n < 1) return fail(TQC_ERR_INVALID, "bad gradient arguments");
    tqc_status st = ensure_cap(cm, n);
    if (st != TQC_OK) return st;
    CM_CUDA(cudaMemcpy(cm->d_X, h_X, sizeof(float) * (size_t)n * cm->n_in, cudaMemcpyHostToDevice), "X");
    CM_CUDA(cudaMemcpy(cm->d_t, h_t, sizeof(float) * n, cudaMemcpyHostToDevice), "t");
    forward(cm, n, 0);
    backward(cm, n, 0);
    CM_CUDA(cudaGetLastError(), "gradient kernels");
    if (h_grad) CM_CUDA(cudaMemcpy(h_grad, cm->d_grad, sizeof(float) * cm->n_params, cudaMemcpyDeviceToHost), "grad");
    if (h_loss) CM_CUDA(cudaMemcpy(h_loss, cm->d_loss, sizeof(float), cudaMemcpyDeviceToHost), "loss");
    return TQC_OK;
}

tqc_status tqc_costmodel_train(tqc_costmodel_t cm, const float *h_X, const float *h_logt, int32_t n, int32_t epochs,
                               int32_t batch, float lr, uint64_t seed, float *final_loss) {
    if (!cm || !h_X || !h_logt || n < 2 || epochs < 1 || batch < 1) return fail(TQC_ERR_INVALID, "bad training arguments");
    const int F = cm->n_in;
    batch = std::min(batch, n);
    // standardise features and labels (statistics kept with the model)
    for (int f = 0; f < F; ++f) {
        double s = 0, s2 = 0;
        for (int i = 0; i < n; ++i) {
            s += h_X[(size_t)i * F + f];
            s2 += (double)h_X[(size_t)i * F + f] * h_X[(size_t)i * F + f];
        }
        const double mu = s / n, var = std::max(s2 / n - mu * mu, 0.0);
        cm->mean[f] = (float)mu;
        cm->stdv[f] = (float)(var > 1e-12 ? std::sqrt(var) : 1.0);
    }
    double s = 0, s2 = 0;
    for (int i = 0; i < n; ++i) {
        s += h_logt[i];
        s2 += (double)h_logt[i] * h_logt[i];
    }
    cm->t_mean = (float)(s / n);
    cm->t_std = (float)std::max(std::sqrt(std::max(s2 / n - (s / n) * (s / n), 0.0)), 1e-6);
    std::vector<float> Xs((size_t)n * F), ts(n);
    for (int i = 0; i < n; ++i) {
        for (int f = 0; f < F; ++f) Xs[(size_t)i * F + f] = (h_X[(size_t)i * F + f] - cm->mean[f]) / cm->stdv[f];
        ts[i] = (h_logt[i] - cm->t_mean) / cm->t_std;
    }
    float *d_allX = nullptr, *d_allt = nullptr;
    int *d_idx = nullptr;
    if (cudaMalloc(&d_allX, sizeof(float) * Xs.size()) != cudaSuccess ||
        cudaMalloc(&d_allt, sizeof(float) * n) != cudaSuccess || cudaMalloc(&d_idx, sizeof(int) * n) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_allX);
        cudaFree(d_allt);
        return fail(TQC_ERR_OOM, "training data");
    }
    tqc_status st = ensure_cap(cm, batch);
    cudaMemcpy(d_allX, Xs.data(), sizeof(float) * Xs.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(d_allt, ts.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
    std::vector<int> idx(n);
    uint64_t rs = seed;
    float last = 0.f;
    const int grid_adam = (int)std::min<int64_t>((cm->n_params + 255) / 256, 1024);
    for (int ep = 0; ep < epochs && st == TQC_OK; ++ep) {
        for (int i = 0; i < n; ++i) idx[i] = i;
        for (int i = n - 1; i > 0; --i) std::swap(idx[i], idx[(int)(uniform01(rs) * (i + 1)) % (i + 1)]);
        cudaMemcpy(d_idx, idx.data(), sizeof(int) * n, cudaMemcpyHostToDevice);
        double ep_loss = 0;
        int nb = 0;
        for (int b0 = 0; b0 + batch <= n; b0 += batch, ++nb) {
            mlp_gather<<<batch, 32>>>(d_allX, d_allt, d_idx + b0, cm->d_X, cm->d_t, batch, F);
            forward(cm, batch, 0);
            backward(cm, batch, 0);
            ++cm->adam_step;
            const float c1 = 1.f - std::pow(0.9f, (float)cm->adam_step);
            const float c2 = 1.f - std::pow(0.999f, (float)cm->adam_step);
            mlp_adam<<<grid_adam, 256>>>(cm->d_theta, cm->d_grad, cm->d_m, cm->d_v, cm->n_params, lr, 0.9f, 0.999f,
                                         1e-8f, c1, c2);
            float l = 0.f;
            cudaMemcpy(&l, cm->d_loss, sizeof(float), cudaMemcpyDeviceToHost);
            ep_loss += l;
        }
        if (cudaGetLastError() != cudaSuccess) st = fail(TQC_ERR_CUDA, "training kernels");
        last = nb ? (float)(ep_loss / nb) : 0.f;
    }
    cudaFree(d_allX);
    cudaFree(d_allt);
    cudaFree(d_idx);
    if (final_loss) *final_loss = last;
    return st;
}

tqc_status tqc_costmodel_predict(tqc_costmodel_t cm, const float *h_X, int32_t n, float *h_logt) {
    if (!cm || !h_X || !h_logt || n < 1) return fail(TQC_ERR_INVALID, "bad prediction arguments");
    return costmodel_predict_host(cm, h_X, n, h_logt);
}

tqc_status tqc_costmodel_save(tqc_costmodel_t cm, const char *path) {
    if (!cm || !path) return fail(TQC_ERR_INVALID, "NULL argument");
    std::vector<float> th(cm->n_params);
    CM_CUDA(cudaMemcpy(th.data(), cm->d_theta, sizeof(float) * cm->n_params, cudaMemcpyDeviceToHost), "save");
    std::ofstream f(path, std::ios::binary);
    if (!f) return fail(TQC_ERR_INVALID, std::string("cannot write ") + path);
    const char magic[8] = {'T', 'Q', 'C', 'M', 'L', 'P', '0', '1'};
    f.write(magic, 8);
    int32_t F = cm->n_in;
    f.write((const char *)&F, 4);
    f.write((const char *)cm->mean.data(), 4 * F);
    f.write((const char *)cm->stdv.data(), 4 * F);
    f.write((const char *)&cm->t_mean, 4);
    f.write((const char *)&cm->t_std, 4);
    f.write((const char *)th.data(), 4 * th.size());
    return f ? TQC_OK : fail(TQC_ERR_INVALID, "write failed");
}

tqc_status tqc_costmodel_load(const char *path, tqc_costmodel_t *out) {
    if (!path || !out) return fail(TQC_ERR_INVALID, "NULL argument");
    *out = nullptr;
    std::ifstream f(path, std::ios::binary);
    if (!f) return fail(TQC_ERR_INVALID, std::string("cannot read ") + path);
    char magic[8];
    int32_t F = 0;
    f.read(magic, 8);
    f.read((char *)&F, 4);
    if (!f || std::memcmp(magic, "TQCMLP01", 8) != 0 || F < 1 || F > 4096)
        return fail(TQC_ERR_INVALID, "not a cost-model file");
    tqc_costmodel_t cm = nullptr;
    tqc_status st = tqc_costmodel_create(F, 0, &cm);
    if (st != TQC_OK) return st;
    f.read((char *)cm->mean.data(), 4 * F);
    f.read((char *)cm->stdv.data(), 4 * F);
    f.read((char *)&cm->t_mean, 4);
    f.read((char *)&cm->t_std, 4);
    std::vector<float> th(cm->n_params);
    f.read((char *)th.data(), 4 * th.size());
    if (!f) {
        tqc_costmodel_destroy(cm);
        return fail(TQC_ERR_INVALID, "truncated cost-model file");
    }
    cudaMemcpy(cm->d_theta, th.data(), 4 * th.size(), cudaMemcpyHostToDevice);
    *out = cm;
    return TQC_OK;
}

}  // extern "C"

namespace tqc {

// standardise, forward on the GPU, un-standardise
tqc_status costmodel_predict_host(tqc_costmodel *cm, const float *h_X, int n, float *h_y) {
    tqc_status st = ensure_cap(cm, n);
    if (st != TQC_OK) return st;
    const int F = cm->n_in;
    std::vector<float> Xs((size_t)n * F);
    for (int i = 0; i < n; ++i)
        for (int f = 0; f < F; ++f) Xs[(size_t)i * F + f] = (h_X[(size_t)i * F + f] - cm->mean[f]) / cm->stdv[f];
    CM_CUDA(cudaMemcpy(cm->d_X, Xs.data(), sizeof(float) * Xs.size(), cudaMemcpyHostToDevice), "X");
    forward(cm, n, 0);
    CM_CUDA(cudaGetLastError(), "forward");
    CM_CUDA(cudaMemcpy(h_y, cm->d_y, sizeof(float) * n, cudaMemcpyDeviceToHost), "y");
    for (int i = 0; i < n; ++i) h_y[i] = h_y[i] * cm->t_std + cm->t_mean;
    return TQC_OK;
}

int costmodel_n_in(tqc_costmodel *cm) { return cm->n_in; }

// Learned planner: the model of `path`, loaded once per process.
tqc_status costmodel_for_path(const char *path, tqc_costmodel **out) {
    std::lock_guard<std::mutex> lk(g_load_mu);
    auto it = g_loaded.find(path);
    if (it != g_loaded.end()) {
        *out = it->second;
        return TQC_OK;
    }
    tqc_costmodel *cm = nullptr;
    tqc_status st = tqc_costmodel_load(path, &cm);
    if (st != TQC_OK) return st;
    g_loaded[path] = cm;
    *out = cm;
    return TQC_OK;
}

}  // namespace tqc
