// Heavy state selection (§IV, Alg. heavy_state_selection).
//
// Step 1 runs on the device: for every output state i of subcircuit C_j, the
// L2 norm of its entries over all cut assignments e,
//     ||p_{j,i}|| = sqrt(sum_e T_j[e][i]^2),
// a column reduction of the [4^c][2^o] node tensor (FP64 partial sums, split
// over e when 2^o alone cannot fill the GPU, and then added in a fixed order,
// so equal tensors give bit-identical norms and ties resolve the same way on
// every call).  Step 2 (seed each subcircuit
// with its heaviest state, then add states in descending norm until the
// product of the per-subcircuit counts reaches s_max) orders a few thousand
// numbers and runs on the host.  The selected states become a new network
// whose subcircuit j keeps only those rows (gathered on the device, padded
// with zero rows to a power of two); its outputs are the per-subcircuit
// selection indices, subcircuit 0's bits lowest, so the ordinary plan /
// contract path reconstructs the product set.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "launch.h"
#include "tqc_internal.h"

struct tqc_net {
    tqc::Net n;
};

namespace tqc {
namespace {

// part[y][x] = sum_{e in [e0, e1)} T[e][x]^2 for split y = blockIdx.y
__global__ void hss_sum2_kernel(const void *T, int dtype, int64_t n_x, int64_t e_per, int64_t n_e, double *part) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n_x) return;
    const int64_t e0 = (int64_t)blockIdx.y * e_per;
    const int64_t e1 = e0 + e_per < n_e ? e0 + e_per : n_e;
    double acc = 0.0;
    if (dtype == TQC_F64) {
        const double *t = (const double *)T;
        for (int64_t e = e0; e < e1; ++e) {
            const double v = t[e * n_x + x];
            acc += v * v;
        }
    } else {
        const float *t = (const float *)T;
        for (int64_t e = e0; e < e1; ++e) {
            const double v = (double)t[e * n_x + x];
            acc += v * v;
        }
    }
    part[(int64_t)blockIdx.y * n_x + x] = acc;
}

// norm[x] = sqrt(sum over the splits, in ascending order, of part[y][x])
__global__ void hss_sqrt_kernel(const double *part, int64_t splits, double *norm, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int64_t y = 0; y < splits; ++y) v += part[y * n + i];
        norm[i] = sqrt(v);
    }
}

// out[e][r] = r < count ? T[e][states[r]] : 0   (r < 2^k)
template <typename V>
__global__ void hss_gather_kernel(const V *T, int64_t n_x, int64_t n_e, const int32_t *states, int32_t count, int k,
                                  V *out) {
    const int64_t n_r = (int64_t)1 << k;
    const int64_t total = n_e * n_r;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = i >> k, r = i & (n_r - 1);
        out[i] = r < count ? T[e * n_x + states[r]] : (V)0;
    }
}

tqc_status node_norms(const Node &nd, double *d_norms, cudaStream_t s) {
    const int64_t n_x = (int64_t)1 << nd.out_qubits.size();
    const int64_t n_e = (int64_t)1 << (2 * nd.cut_ids.size());
    const int threads = 256;
    const int64_t xb = (n_x + threads - 1) / threads;
    // split the cut assignments so that about four CTAs per SM run
    int64_t ys = std::max<int64_t>(1, std::min<int64_t>(n_e, (4ll * sm_count() + xb - 1) / xb));
    ys = std::min<int64_t>(ys, 65535);
    const int64_t e_per = (n_e + ys - 1) / ys;
    ys = (n_e + e_per - 1) / e_per;
    if (xb > 2147483647ll) return fail(TQC_ERR_UNSUPPORTED, "hss: too many output states");
    // one split: the partial sums are the norms' squares, in place; several:
    // stream-ordered scratch of splits x 2^o partial sums (at most a few MB)
    double *part = d_norms;
    if (ys > 1 && cudaMallocAsync((void **)&part, sizeof(double) * (size_t)(ys * n_x), s) != cudaSuccess) {
        cudaGetLastError();
        return fail(TQC_ERR_OOM, "hss: partial sums");
    }
    hss_sum2_kernel<<<dim3((unsigned)xb, (unsigned)ys), threads, 0, s>>>(nd.d_data, nd.dtype, n_x, e_per, n_e, part);
    const int64_t sb = std::min<int64_t>((n_x + threads - 1) / threads, 16ll * sm_count());
    hss_sqrt_kernel<<<(unsigned)sb, threads, 0, s>>>(part, ys, d_norms, n_x);
    cudaError_t e = cudaGetLastError();
    if (ys > 1) cudaFreeAsync(part, s);
    if (e != cudaSuccess) return fail(TQC_ERR_CUDA, "hss: norm kernels");
    return TQC_OK;
}

}  // namespace
}  // namespace tqc

using namespace tqc;

extern "C" {

tqc_status tqc_hss_norms(tqc_net_t net, int32_t sub, double *d_norms, void *cuda_stream) {
    if (!net || !d_norms) return fail(TQC_ERR_INVALID, "NULL argument");
    Net &n = net->n;
    if (!n.has_data) return fail(TQC_ERR_INVALID, "shape-only network has no device tensors");
    if (sub < 0 || sub >= (int)n.nodes.size()) return fail(TQC_ERR_INVALID, "subcircuit index out of range");
    return node_norms(n.nodes[(size_t)sub], d_norms, (cudaStream_t)cuda_stream);
}

tqc_status tqc_hss_select(tqc_net_t net, int64_t s_max, int32_t *counts, int32_t *states, int64_t states_cap,
                          int64_t *n_states_out) {
    if (!net || !counts || !states || !n_states_out) return fail(TQC_ERR_INVALID, "NULL argument");
    if (s_max < 1) return fail(TQC_ERR_INVALID, "s_max must be at least 1");
    Net &n = net->n;
    if (!n.has_data) return fail(TQC_ERR_INVALID, "shape-only network has no device tensors");
    const int m = (int)n.nodes.size();
    // step 1 on the device: every subcircuit's state norms
    std::vector<std::vector<double>> norms(m);
    size_t biggest = 0;
    for (auto &nd : n.nodes) biggest = std::max(biggest, (size_t)1 << nd.out_qubits.size());
    double *d = nullptr;
    if (cudaMalloc(&d, sizeof(double) * biggest) != cudaSuccess) {
        cudaGetLastError();
        return fail(TQC_ERR_OOM, "hss: norm buffer");
    }
    for (int j = 0; j < m; ++j) {
        const size_t nx = (size_t)1 << n.nodes[j].out_qubits.size();
        tqc_status st = node_norms(n.nodes[j], d, 0);
        if (st != TQC_OK) {
            cudaFree(d);
            return st;
        }
        norms[j].resize(nx);
        if (cudaMemcpy(norms[j].data(), d, sizeof(double) * nx, cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaFree(d);
            return fail(TQC_ERR_CUDA, "hss: norm copy");
        }
    }
    cudaFree(d);
    // step 2: seed every subcircuit with its heaviest state (ties: lowest
    // index), then take states in descending norm (ties: lowest subcircuit,
    // then lowest index) while the product of the counts is below s_max
    std::vector<std::vector<int32_t>> sel(m);
    struct Cand {
        double v;
        int32_t j, i;
    };
    std::vector<Cand> pool;
    for (int j = 0; j < m; ++j) {
        const auto &v = norms[j];
        const int32_t best = (int32_t)(std::max_element(v.begin(), v.end()) - v.begin());
        sel[j].push_back(best);
        for (int32_t i = 0; i < (int32_t)v.size(); ++i)
            if (i != best) pool.push_back({v[i], j, i});
    }
    std::stable_sort(pool.begin(), pool.end(), [](const Cand &a, const Cand &b) {
        if (a.v != b.v) return a.v > b.v;
        if (a.j != b.j) return a.j < b.j;
        return a.i < b.i;
    });
    auto product = [&]() {
        double p = 1.0;
        for (auto &x : sel) p *= (double)x.size();
        return p;
    };
    for (size_t k = 0; k < pool.size() && product() < (double)s_max; ++k) sel[pool[k].j].push_back(pool[k].i);
    int64_t total = 0;
    for (int j = 0; j < m; ++j) total += (int64_t)sel[j].size();
    if (total > states_cap) return fail(TQC_ERR_INVALID, "hss: states buffer too small (" + std::to_string(total) + ")");
    int64_t off = 0;
    for (int j = 0; j < m; ++j) {
        std::sort(sel[j].begin(), sel[j].end());
        counts[j] = (int32_t)sel[j].size();
        std::copy(sel[j].begin(), sel[j].end(), states + off);
        off += (int64_t)sel[j].size();
    }
    *n_states_out = (int64_t)product();
    return TQC_OK;
}

tqc_status tqc_network_select(tqc_net_t net, const int32_t *counts, const int32_t *states, tqc_net_t *out) {
    if (!net || !counts || !states || !out) return fail(TQC_ERR_INVALID, "NULL argument");
    *out = nullptr;
    const Net &src = net->n;
    if (!src.has_data) return fail(TQC_ERR_INVALID, "shape-only network has no device tensors");
    const int m = (int)src.nodes.size();
    Net dst;
    dst.n_cuts = src.n_cuts;
    dst.cut_nodes = src.cut_nodes;
    dst.has_data = true;
    dst.device = src.device;
    std::vector<int> kbits(m);
    int nq = 0, off = 0;
    for (int j = 0; j < m; ++j) {
        const int64_t nx = (int64_t)1 << src.nodes[j].out_qubits.size();
        if (counts[j] < 1 || counts[j] > nx)
            return fail(TQC_ERR_INVALID, "subcircuit " + std::to_string(j) + ": count must be in 1.." + std::to_string(nx));
        for (int r = 0; r < counts[j]; ++r) {
            const int32_t st = states[off + r];
            if (st < 0 || st >= nx || (r > 0 && st <= states[off + r - 1]))
                return fail(TQC_ERR_INVALID, "subcircuit " + std::to_string(j) + ": states must be increasing and in range");
        }
        int k = 0;
        while (((int64_t)1 << k) < counts[j]) ++k;
        kbits[j] = k;
        nq += k;
        off += counts[j];
    }
    if (nq == 0) kbits[0] = nq = 1;  // one padding bit: the network needs at least one output
    if (nq > 128) return fail(TQC_ERR_UNSUPPORTED, "selection has more than 128 index bits");
    dst.n_qubits = nq;
    int q = 0;
    off = 0;
    for (int j = 0; j < m; ++j) {
        const Node &sn = src.nodes[j];
        Node nd;
        nd.cut_ids = sn.cut_ids;
        nd.cut_role = sn.cut_role;
        nd.dtype = sn.dtype;
        for (int b = 0; b < kbits[j]; ++b) nd.out_qubits.push_back(q++);
        const int64_t n_e = (int64_t)1 << (2 * sn.cut_ids.size());
        nd.elems = n_e << kbits[j];
        const size_t esz = sn.dtype == TQC_F64 ? 8 : 4;
        int32_t *d_states = nullptr;
        cudaError_t e = cudaMalloc(&nd.d_data, (size_t)nd.elems * esz);
        if (e == cudaSuccess) e = cudaMalloc(&d_states, sizeof(int32_t) * counts[j]);
        if (e == cudaSuccess)
            e = cudaMemcpy(d_states, states + off, sizeof(int32_t) * counts[j], cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            const int64_t nx = (int64_t)1 << sn.out_qubits.size();
            const int64_t blocks = std::min<int64_t>((nd.elems + 255) / 256, 16ll * sm_count());
            if (sn.dtype == TQC_F64)
                hss_gather_kernel<double><<<(unsigned)blocks, 256>>>((const double *)sn.d_data, nx, n_e, d_states,
                                                                     counts[j], kbits[j], (double *)nd.d_data);
            else
                hss_gather_kernel<float><<<(unsigned)blocks, 256>>>((const float *)sn.d_data, nx, n_e, d_states,
                                                                    counts[j], kbits[j], (float *)nd.d_data);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
        }
        cudaFree(d_states);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaFree(nd.d_data);
            for (auto &x : dst.nodes) cudaFree(x.d_data);
            return fail(TQC_ERR_CUDA, std::string("network_select: ") + cudaGetErrorString(e));
        }
        dst.nodes.push_back(std::move(nd));
        off += counts[j];
    }
    struct tqc_net *h = new (std::nothrow) struct tqc_net;
    if (!h) {
        for (auto &x : dst.nodes) cudaFree(x.d_data);
        return fail(TQC_ERR_OOM, "host allocation failed");
    }
    h->n = std::move(dst);
    *out = h;
    return TQC_OK;
}

}  // extern "C"
