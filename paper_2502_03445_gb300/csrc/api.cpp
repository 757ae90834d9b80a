// C ABI of libtqc: argument checking, network IR construction and handle
// management.  Device work lives in executor.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>

#include "tqc_internal.h"

struct tqc_net {
    tqc::Net n;
};
struct tqc_plan {
    tqc::Plan p;
};

namespace tqc {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

tqc_status fail(tqc_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

}  // namespace tqc

using namespace tqc;

extern "C" {

const char *tqc_last_error(void) { return g_err.c_str(); }

void tqc_plan_opts_default(tqc_plan_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = TQC_PREC_AUTO;
    o->planner = TQC_PLANNER_AUTO;
}

tqc_status tqc_network_create(int32_t n_qubits, int32_t n_sub, const tqc_subcircuit *subs, tqc_net_t *out) {
    if (!out) return fail(TQC_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (n_qubits < 1 || n_qubits > 128) return fail(TQC_ERR_INVALID, "n_qubits must be in 1..128");
    if (n_sub < 1 || n_sub > 63) return fail(TQC_ERR_INVALID, "n_sub must be in 1..63");
    if (!subs) return fail(TQC_ERR_INVALID, "subs is NULL");
    Net net;
    net.n_qubits = n_qubits;
    std::vector<int> q_owner(n_qubits, -1);
    int max_cut = -1;
    int with_data = 0;
    for (int j = 0; j < n_sub; ++j) {
        const tqc_subcircuit &s = subs[j];
        std::string who = "subcircuit " + std::to_string(j);
        if (s.n_out < 0 || s.n_out > 40) return fail(TQC_ERR_INVALID, who + ": n_out must be in 0..40");
        if (s.n_cut < 0 || s.n_cut > 20) return fail(TQC_ERR_INVALID, who + ": n_cut must be in 0..20");
        if (s.n_out + 2 * s.n_cut > 46) return fail(TQC_ERR_UNSUPPORTED, who + ": tensor larger than 2^46 elements");
        if ((s.n_out && !s.out_qubits) || (s.n_cut && (!s.cut_ids || !s.cut_role)))
            return fail(TQC_ERR_INVALID, who + ": NULL label array");
        Node nd;
        for (int k = 0; k < s.n_out; ++k) {
            int q = s.out_qubits[k];
            if (q < 0 || q >= n_qubits) return fail(TQC_ERR_INVALID, who + ": output qubit " + std::to_string(q) + " out of range");
            if (q_owner[q] >= 0)
                return fail(TQC_ERR_INVALID, who + ": output qubit " + std::to_string(q) + " already output by subcircuit " +
                                                 std::to_string(q_owner[q]));
            q_owner[q] = j;
            nd.out_qubits.push_back(q);
        }
        for (int d = 0; d < s.n_cut; ++d) {
            int c = s.cut_ids[d];
            if (c < 0 || c > 62) return fail(TQC_ERR_INVALID, who + ": cut id " + std::to_string(c) + " out of range 0..62");
            if (s.cut_role[d] != 0 && s.cut_role[d] != 1)
                return fail(TQC_ERR_INVALID, who + ": cut " + std::to_string(c) + " role must be 0 or 1");
            if (std::find(nd.cut_ids.begin(), nd.cut_ids.end(), c) != nd.cut_ids.end())
                return fail(TQC_ERR_INVALID, who + ": cut " + std::to_string(c) + " joins a subcircuit to itself");
            nd.cut_ids.push_back(c);
            nd.cut_role.push_back(s.cut_role[d]);
            max_cut = std::max(max_cut, c);
        }
        if (s.data) {
            ++with_data;
            if (s.dtype != TQC_F64 && s.dtype != TQC_F32) return fail(TQC_ERR_INVALID, who + ": dtype must be TQC_F64 or TQC_F32");
        }
        nd.dtype = s.dtype;
        nd.elems = (int64_t)1 << (s.n_out + 2 * s.n_cut);
        net.nodes.push_back(std::move(nd));
    }
    for (int q = 0; q < n_qubits; ++q)
        if (q_owner[q] < 0) return fail(TQC_ERR_INVALID, "qubit " + std::to_string(q) + " is not an output of any subcircuit");
    net.n_cuts = max_cut + 1;
    net.cut_nodes.assign(net.n_cuts, {-1, -1});
    for (int j = 0; j < n_sub; ++j) {
        const Node &nd = net.nodes[j];
        for (size_t d = 0; d < nd.cut_ids.size(); ++d) {
            int c = nd.cut_ids[d], r = nd.cut_role[d];
            if (net.cut_nodes[c][r] >= 0)
                return fail(TQC_ERR_INVALID, "cut " + std::to_string(c) + ": two " + (r ? "downstream" : "upstream") +
                                                 " ends (subcircuits " + std::to_string(net.cut_nodes[c][r]) + " and " +
                                                 std::to_string(j) + ")");
            net.cut_nodes[c][r] = j;
        }
    }
    for (int c = 0; c < net.n_cuts; ++c)
        if (net.cut_nodes[c][0] < 0 || net.cut_nodes[c][1] < 0)
            return fail(TQC_ERR_INVALID, "cut " + std::to_string(c) + ": missing " +
                                             (net.cut_nodes[c][0] < 0 ? "upstream" : "downstream") + " end");
    if (with_data != 0 && with_data != n_sub)
        return fail(TQC_ERR_INVALID, "either every subcircuit or none carries data");
    net.has_data = with_data == n_sub;
    if (net.has_data) {
        if (cudaGetDevice(&net.device) != cudaSuccess) return fail(TQC_ERR_CUDA, "no CUDA device");
        for (int j = 0; j < n_sub; ++j) {
            Node &nd = net.nodes[j];
            size_t bytes = (size_t)nd.elems * (nd.dtype == TQC_F64 ? 8 : 4);
            cudaError_t e = cudaMalloc(&nd.d_data, bytes);
            if (e != cudaSuccess) {
                for (auto &x : net.nodes) cudaFree(x.d_data);
                cudaGetLastError();
                return fail(TQC_ERR_OOM, "subcircuit " + std::to_string(j) + ": device allocation of " +
                                             std::to_string(bytes) + " bytes failed");
            }
            e = cudaMemcpy(nd.d_data, subs[j].data, bytes, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                for (auto &x : net.nodes) cudaFree(x.d_data);
                return fail(TQC_ERR_CUDA, std::string("tensor upload: ") + cudaGetErrorString(e));
            }
        }
    }
    struct tqc_net *h = new (std::nothrow) struct tqc_net;
    if (!h) {
        for (auto &x : net.nodes) cudaFree(x.d_data);
        return fail(TQC_ERR_OOM, "host allocation failed");
    }
    h->n = std::move(net);
    *out = h;
    return TQC_OK;
}

tqc_status tqc_network_upload(tqc_net_t net, int32_t sub, int32_t dtype, const void *host_data, void *stream) {
    if (!net || !host_data) return fail(TQC_ERR_INVALID, "NULL argument");
    Net &n = net->n;
    if (!n.has_data) return fail(TQC_ERR_INVALID, "shape-only network has no device tensors");
    if (sub < 0 || sub >= (int)n.nodes.size()) return fail(TQC_ERR_INVALID, "subcircuit index out of range");
    Node &nd = n.nodes[sub];
    if (dtype != nd.dtype) return fail(TQC_ERR_INVALID, "upload dtype differs from the network's");
    size_t bytes = (size_t)nd.elems * (nd.dtype == TQC_F64 ? 8 : 4);
    cudaError_t e = cudaMemcpyAsync(nd.d_data, host_data, bytes, cudaMemcpyHostToDevice, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(TQC_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
    n.version++;
    return TQC_OK;
}

tqc_status tqc_destroy(tqc_net_t net) {
    if (!net) return fail(TQC_ERR_INVALID, "NULL network");
    if (net->n.live_plans > 0) return fail(TQC_ERR_INVALID, "network still has live plans");
    for (auto &nd : net->n.nodes)
        if (nd.d_data) cudaFree(nd.d_data);
    delete net;
    return TQC_OK;
}

tqc_status tqc_plan(tqc_net_t net, const tqc_plan_opts *opts, tqc_plan_t *out) {
    if (!net || !out) return fail(TQC_ERR_INVALID, "NULL argument");
    *out = nullptr;
    tqc_plan_opts o;
    tqc_plan_opts_default(&o);
    if (opts) o = *opts;
    struct tqc_plan *h = new (std::nothrow) struct tqc_plan;
    if (!h) return fail(TQC_ERR_OOM, "host allocation failed");
    tqc_status st;
    try {
        st = build_plan(&net->n, o, &h->p);
    } catch (const std::bad_alloc &) {
        st = fail(TQC_ERR_OOM, "host allocation failed while planning");
    } catch (const std::exception &ex) {
        st = fail(TQC_ERR_INVALID, std::string("planning failed: ") + ex.what());
    }
    if (st != TQC_OK) {
        delete h;
        return st;
    }
    net->n.live_plans++;
    *out = h;
    return TQC_OK;
}

tqc_status tqc_plan_info(tqc_plan_t plan, double *flops, double *bytes, int32_t *n_slices, int32_t *n_steps) {
    if (!plan) return fail(TQC_ERR_INVALID, "NULL plan");
    const Plan &p = plan->p;
    if (flops) *flops = p.flops;
    if (bytes) *bytes = p.bytes;
    if (n_slices) *n_slices = (int32_t)p.n_slices();
    if (n_steps) *n_steps = (int32_t)p.steps.size();
    return TQC_OK;
}

tqc_status tqc_plan_step(tqc_plan_t plan, int32_t step, int32_t *lm, int32_t *ln, int32_t *lk, int32_t *klass,
                         int32_t *prec) {
    if (!plan) return fail(TQC_ERR_INVALID, "NULL plan");
    const Plan &p = plan->p;
    if (step < 0 || step >= (int)p.steps.size()) return fail(TQC_ERR_INVALID, "step out of range");
    const StepPlan &s = p.steps[step];
    if (lm) *lm = s.mb;
    if (ln) *ln = s.nb;
    if (lk) *lk = s.kb;
    if (klass) *klass = s.klass;
    if (prec) *prec = s.klass == KC_UMMA ? s.prec : TQC_PREC_FP32;
    return TQC_OK;
}

int32_t tqc_plan_describe(tqc_plan_t plan, char *buf, int32_t size) {
    if (!plan) return -1;
    plan->p.describe_json = plan_describe(plan->p);
    const std::string &s = plan->p.describe_json;
    if (buf && size > 0) {
        size_t n = std::min((size_t)size - 1, s.size());
        std::memcpy(buf, s.data(), n);
        buf[n] = 0;
    }
    return (int32_t)s.size();
}

tqc_status tqc_contract(tqc_plan_t plan, const uint8_t *fixed_bits, void *d_out, int32_t out_dtype, double *z_out,
                        void *stream) {
    if (!plan) return fail(TQC_ERR_INVALID, "NULL plan");
    if (!d_out) return fail(TQC_ERR_INVALID, "d_out is NULL");
    if (out_dtype != TQC_F32 && out_dtype != TQC_F64) return fail(TQC_ERR_INVALID, "out_dtype must be TQC_F32 or TQC_F64");
    if (!plan->p.net->has_data) return fail(TQC_ERR_INVALID, "shape-only network cannot be contracted");
    return exec_contract(&plan->p, fixed_bits, d_out, out_dtype, z_out, stream);
}

tqc_status tqc_contract_states(tqc_plan_t plan, const uint64_t *states, int64_t n_states, void *d_out,
                               int32_t out_dtype, double *z_out, void *stream) {
    if (!plan) return fail(TQC_ERR_INVALID, "NULL plan");
    if (n_states > 0 && (!states || !d_out)) return fail(TQC_ERR_INVALID, "NULL states or d_out");
    if (out_dtype != TQC_F32 && out_dtype != TQC_F64) return fail(TQC_ERR_INVALID, "out_dtype must be TQC_F32 or TQC_F64");
    if (!plan->p.net->has_data) return fail(TQC_ERR_INVALID, "shape-only network cannot be contracted");
    try {
        return exec_contract_states(&plan->p, states, n_states, d_out, out_dtype, z_out, stream);
    } catch (const std::bad_alloc &) {
        return fail(TQC_ERR_OOM, "host allocation failed");
    }
}

tqc_status tqc_contract_host(tqc_plan_t plan, const void *const *host_tensors, int32_t in_dtype, void *host_out,
                             int32_t out_dtype, double *z_out, void *stream) {
    if (!plan || !host_out) return fail(TQC_ERR_INVALID, "NULL argument");
    if (out_dtype != TQC_F32 && out_dtype != TQC_F64) return fail(TQC_ERR_INVALID, "out_dtype must be TQC_F32 or TQC_F64");
    Plan &p = plan->p;
    if (!p.net->has_data) return fail(TQC_ERR_INVALID, "shape-only network cannot be contracted");
    cudaStream_t s = (cudaStream_t)stream;
    if (host_tensors)
        for (int j = 0; j < p.m; ++j)
            if (host_tensors[j]) {
                Node &nd = p.net->nodes[j];
                if (in_dtype != nd.dtype) return fail(TQC_ERR_INVALID, "in_dtype differs from the network's");
                size_t bytes = (size_t)nd.elems * (nd.dtype == TQC_F64 ? 8 : 4);
                cudaError_t e = cudaMemcpyAsync(nd.d_data, host_tensors[j], bytes, cudaMemcpyHostToDevice, s);
                if (e != cudaSuccess) return fail(TQC_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
                p.net->version++;
            }
    int64_t ob = p.out_elems() * (out_dtype == TQC_F64 ? 8 : 4);
    // Pinned host memory mapped into the device's address space (Grace's
    // memory over NVLink-C2C): the last kernel stores the probabilities there
    // directly, with no device copy of the result and no separate download.
    {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, host_out) == cudaSuccess && at.type == cudaMemoryTypeHost &&
            at.devicePointer != nullptr) {
            tqc_status st = exec_contract(&p, nullptr, at.devicePointer, out_dtype, nullptr, stream);
            if (st != TQC_OK) return st;
            cudaError_t e = cudaSuccess;
            if (z_out) e = cudaMemcpyAsync(z_out, p.d_zinfo, sizeof(double), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return fail(TQC_ERR_CUDA, std::string("result: ") + cudaGetErrorString(e));
            return TQC_OK;
        }
        cudaGetLastError();
    }
    if (p.d_hostout_bytes < ob) {
        if (p.d_hostout) cudaFree(p.d_hostout);
        p.d_hostout = nullptr;
        p.d_hostout_bytes = 0;
        if (cudaMalloc(&p.d_hostout, ob) != cudaSuccess) {
            cudaGetLastError();
            return fail(TQC_ERR_OOM, "device output buffer");
        }
        p.d_hostout_bytes = ob;
    }
    tqc_status st = exec_contract(&p, nullptr, p.d_hostout, out_dtype, nullptr, stream);
    if (st != TQC_OK) return st;
    cudaError_t e = cudaMemcpyAsync(host_out, p.d_hostout, ob, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && z_out) e = cudaMemcpyAsync(z_out, p.d_zinfo, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(TQC_ERR_CUDA, std::string("result download: ") + cudaGetErrorString(e));
    return TQC_OK;
}

tqc_status tqc_plan_features(tqc_plan_t plan, float *out, int32_t n) {
    if (!plan || !out) return fail(TQC_ERR_INVALID, "NULL argument");
    if (n < TQC_PLAN_FEATURES) return fail(TQC_ERR_INVALID, "feature buffer smaller than TQC_PLAN_FEATURES");
    std::vector<double> f = plan_features(plan->p);
    for (int i = 0; i < TQC_PLAN_FEATURES; ++i) out[i] = i < (int)f.size() ? (float)f[i] : 0.f;
    return TQC_OK;
}

tqc_status tqc_plan_candidates(tqc_net_t net, const tqc_plan_opts *opts, int32_t max_n, int32_t *orders,
                               int32_t *n_out) {
    if (!net || !orders || !n_out || max_n < 1) return fail(TQC_ERR_INVALID, "bad candidate arguments");
    tqc_plan_opts o;
    tqc_plan_opts_default(&o);
    if (opts) o = *opts;
    std::vector<std::vector<int32_t>> c;
    try {
        c = plan_candidate_orders(&net->n, o, max_n);
    } catch (const std::exception &ex) {
        return fail(TQC_ERR_INVALID, std::string("candidates: ") + ex.what());
    }
    const int per = 2 * ((int)net->n.nodes.size() - 1);
    int k = 0;
    for (auto &ord : c) {
        if (k >= max_n) break;
        std::copy(ord.begin(), ord.end(), orders + (size_t)k * per);
        ++k;
    }
    *n_out = k;
    return TQC_OK;
}


tqc_status tqc_plan_profile(tqc_plan_t plan, int32_t enable) {
    if (!plan) return fail(TQC_ERR_INVALID, "NULL plan");
    if (!enable) exec_clear_events(&plan->p);
    plan->p.profile = enable ? 1 : 0;
    return TQC_OK;
}

tqc_status tqc_plan_step_time(tqc_plan_t plan, int32_t step, double *mean_ms, int32_t *launches) {
    if (!plan) return fail(TQC_ERR_INVALID, "NULL plan");
    if (step < 0 || step >= (int)plan->p.steps.size()) return fail(TQC_ERR_INVALID, "step out of range");
    int n = 0;
    tqc_status st = exec_step_time(&plan->p, step, mean_ms, &n);
    if (launches) *launches = n;
    return st;
}

tqc_status tqc_plan_destroy(tqc_plan_t plan) {
    if (!plan) return fail(TQC_ERR_INVALID, "NULL plan");
    exec_release(&plan->p);
    if (plan->p.d_hostout) cudaFree(plan->p.d_hostout);
    plan->p.net->live_plans--;
    delete plan;
    return TQC_OK;
}

}  // extern "C"
