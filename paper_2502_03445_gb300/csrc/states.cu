// Reconstruction of an arbitrary list of states.
//
// §VII-C measures the time to reconstruct one million arbitrary output
// states.  For one state x, Eq. reconstruction is a scalar network: node j
// contributes the 4^{c_j} values T_j[.][x|out_j], and the plan's pairwise
// steps over the cut indices alone (a plan with no free qubits) contract it.
//
// Two forms, chosen from the plan:
//   fused      one persistent kernel; a CTA takes one state at a time and
//              runs every step of the single-state plan in shared memory.
//              Its leaf operands are rows of per-node tables
//              Tt_j[x][cuts] (node tensors transposed so that the 4^{c_j}
//              values a state needs are one contiguous row, FP32, built by
//              the ingest kernel once per tensor version and small enough
//              to stay in L2); intermediates never leave shared memory.
//              Taken when every intermediate fits (e.g. 4^6 floats).
//   per-state  networks whose single-state intermediates are large (the
//              48-qubit QAOA network: 4^12 floats, GEMMs of 2^24..2^28
//              multiply-adds per state) run the single-state plan once per
//              state through the ordinary step kernels, with the state's
//              bits as the fixed bits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "launch.h"

namespace tqc {

namespace {

constexpr int ST_THREADS = 256;
constexpr int ST_MAX_LEAVES = 16;
constexpr int ST_MAX_STEPS = ST_MAX_LEAVES - 1;
constexpr int ST_MAX_SMEM_FLOATS = 200 * 1024 / 4;

struct SLeaf {
    const float *table;  // [2^{n_q}][4^{cuts}]: row x is the leaf operand of states with x|out_j = x
    int32_t row_log2;    // log2 of the row length (2 * cuts)
    int32_t q_off, n_q;  // output qubits in SProgram::qubits[q_off .. q_off + n_q): bit k of x
};

struct SStep {
    int32_t a_src, b_src;   // >= 0: leaf index; < 0: result of step (-1 - src)
    int32_t mb, nb, kb;     // log2 of M, N, K
    uint32_t maskR, maskC;  // result-layout bits of the row / column index bits
    int32_t c_kb;           // log2 K of the step consuming the result; -1 for the final step
    int32_t c_off;          // shared-memory offset (floats) of the result: rows of 2^c_kb, padded
    int32_t a_off, b_off;   // shared-memory offsets of the operands
    int32_t tm, tn;         // register tile of a thread (rows strided by M / tm, columns by N / tn)
    int32_t ksplit;         // K ranges of one output tile (summed through the reduction buffer)
    int32_t tab_off;        // shared-memory offset of the result offsets of rows (M) then columns (N)
};

struct SProgram {
    int32_t n_leaves, n_steps;
    int8_t qubits[64];
    SLeaf leaf[ST_MAX_LEAVES];
    SStep step[ST_MAX_STEPS];
    int32_t red_off;
    int32_t smem_floats;
};

// Row pitch of a [rows][K] operand in shared memory: K + 4 floats keeps
// float4 access and spreads rows over the banks.
__host__ __device__ __forceinline__ int pitch_of(int k) { return k >= 4 ? k + 4 : k; }

__global__ void __launch_bounds__(ST_THREADS, 3)
    states_kernel(const __grid_constant__ SProgram P, const uint64_t *__restrict__ states, int64_t n, void *out,
                  int out_f64, const double *zinfo) {
    extern __shared__ __align__(16) float sm[];
    __shared__ int64_t proj[ST_MAX_LEAVES];
    const int tid = threadIdx.x;
    const double scale = zinfo[1];
    // Every state runs the same program: the place of result row r and column
    // c in the consumer's padded operand is tab[r] + tab[M + c] (the row and
    // column bits are disjoint, so the deposit of (r, c) splits into two
    // parts), computed once per CTA.
    for (int si = 0; si < P.n_steps; ++si) {
        const SStep &S = P.step[si];
        const int M = 1 << S.mb, N = 1 << S.nb;
        int *tab = (int *)(sm + S.tab_off);
        const int ck = S.c_kb < 0 ? 1 : 1 << S.c_kb, pc = pitch_of(ck);
        for (int i = tid; i < M + N; i += ST_THREADS) {
            const uint32_t d = i < M ? pdep32((uint32_t)i, S.maskR) : pdep32((uint32_t)(i - M), S.maskC);
            tab[i] = S.c_kb < 0 ? 0 : (int)(d >> S.c_kb) * pc + (int)(d & (uint32_t)(ck - 1));
        }
    }
    __syncthreads();
    for (int64_t s = blockIdx.x; s < n; s += gridDim.x) {
        const uint64_t x = states[s];
        if (tid < P.n_leaves) {
            const SLeaf &L = P.leaf[tid];
            int64_t pj = 0;
            for (int k = 0; k < L.n_q; ++k) pj |= (int64_t)((x >> P.qubits[L.q_off + k]) & 1ull) << k;
            proj[tid] = pj;
        }
        __syncthreads();
        if (P.n_steps == 0) {  // one subcircuit without cuts: a table lookup
            if (tid == 0) {
                const double v = (double)P.leaf[0].table[proj[0]] * scale;
                if (out_f64) ((double *)out)[s] = v;
                else ((float *)out)[s] = (float)v;
            }
            __syncthreads();
            continue;
        }
        for (int si = 0; si < P.n_steps; ++si) {
            const SStep &S = P.step[si];
            const int M = 1 << S.mb, N = 1 << S.nb, K = 1 << S.kb;
            const int pk = pitch_of(K);
            // stage leaf operands (rows x K, row-major in the table) into padded rows
#pragma unroll
            for (int op = 0; op < 2; ++op) {
                const int src = op ? S.b_src : S.a_src;
                if (src < 0) continue;
                const int rows = op ? N : M;
                const float *row = P.leaf[src].table + (proj[src] << P.leaf[src].row_log2);
                float *dst = sm + (op ? S.b_off : S.a_off);
                if (K >= 4) {
                    const int lq = S.kb - 2;  // float4s per row: K / 4
                    for (int i = tid; i < rows << lq; i += ST_THREADS) {
                        const int r = i >> lq, k4 = i & ((1 << lq) - 1);
                        *(float4 *)(dst + r * pk + 4 * k4) = __ldg((const float4 *)row + i);
                    }
                } else {
                    for (int i = tid; i < rows * K; i += ST_THREADS) dst[i] = __ldg(row + i);
                }
            }
            __syncthreads();
            const float *A = sm + S.a_off, *B = sm + S.b_off;
            const int tm = S.tm, tn = S.tn;
            const int rstride = M / tm, cstride = N / tn;
            const int lc = __ffs(cstride) - 1, lt = lc + __ffs(rstride) - 1;  // log2 of cstride, n_tiles
            const int n_tiles = rstride * cstride;
            const int kc = K / S.ksplit;
            float *red = sm + P.red_off;
            const int *tab = (const int *)(sm + S.tab_off);
            float *res = sm + S.c_off;
            // result element (r, c) -> its place in the consumer's padded operand
            auto put = [&](int r, int c, float v) {
                if (S.c_kb < 0) {
                    const double d = (double)v * scale;
                    if (out_f64) ((double *)out)[s] = d;
                    else ((float *)out)[s] = (float)d;
                    return;
                }
                res[tab[r] + tab[M + c]] = v;
            };
            for (int u = tid; u < n_tiles * S.ksplit; u += ST_THREADS) {
                const int t = u & (n_tiles - 1), ks = u >> lt;
                const int rt = t >> lc, ct = t & (cstride - 1);
                float acc[4][4];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
                const int k0 = ks * kc;
                if (kc >= 4) {
                    for (int k = k0; k < k0 + kc; k += 4) {
                        float4 a[4], b[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            if (i < tm) a[i] = *(const float4 *)(A + (rt + i * rstride) * pk + k);
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if (j < tn) b[j] = *(const float4 *)(B + (ct + j * cstride) * pk + k);
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                if (i < tm && j < tn) {
                                    acc[i][j] = fmaf(a[i].x, b[j].x, acc[i][j]);
                                    acc[i][j] = fmaf(a[i].y, b[j].y, acc[i][j]);
                                    acc[i][j] = fmaf(a[i].z, b[j].z, acc[i][j]);
                                    acc[i][j] = fmaf(a[i].w, b[j].w, acc[i][j]);
                                }
                    }
                } else {
                    for (int k = k0; k < k0 + kc; ++k)
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                if (i < tm && j < tn)
                                    acc[i][j] = fmaf(A[(rt + i * rstride) * pk + k], B[(ct + j * cstride) * pk + k],
                                                     acc[i][j]);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (i < tm && j < tn) {
                            const int r = rt + i * rstride, c = ct + j * cstride;
                            if (S.ksplit == 1) put(r, c, acc[i][j]);
                            else red[ks * M * N + r * N + c] = acc[i][j];
                        }
            }
            __syncthreads();
            if (S.ksplit > 1) {
                for (int o = tid; o < M * N; o += ST_THREADS) {
                    float v = 0.f;
                    for (int ks = 0; ks < S.ksplit; ++ks) v += red[ks * M * N + o];
                    put(o / N, o % N, v);
                }
                __syncthreads();
            }
        }
    }
}

int64_t align4(int64_t x) { return (x + 3) & ~int64_t(3); }

// The fused form's program for a single-state plan, without table pointers
// (set at launch); false when the plan does not fit its limits.
bool build_program(const Plan &p, SProgram *P, std::string *why) {
    std::memset(P, 0, sizeof(*P));
    if (!p.free_qubits.empty()) return *why = "free qubits", false;
    if (p.n_slices() != 1) return *why = "sliced", false;
    if (p.m > ST_MAX_LEAVES) return *why = "more than 16 subcircuits", false;
    if (p.net->n_qubits > 64) return *why = "more than 64 qubits", false;
    P->n_leaves = p.m;
    P->n_steps = (int)p.steps.size();
    int q = 0;
    for (int j = 0; j < p.m; ++j) {
        const Node &nd = p.net->nodes[j];
        P->leaf[j].row_log2 = p.tensors[j].nbits();
        P->leaf[j].q_off = q;
        P->leaf[j].n_q = (int)nd.out_qubits.size();
        for (int oq : nd.out_qubits) P->qubits[q++] = (int8_t)oq;
    }
    // shared memory: two staging areas for leaf operands, the reduction
    // buffer, then one region per intermediate
    int64_t stg[2] = {0, 0}, red = 0;
    std::vector<int> consumer(p.tensors.size(), -1);
    for (size_t s = 0; s < p.steps.size(); ++s) {
        consumer[(size_t)p.steps[s].a] = (int)s;
        consumer[(size_t)p.steps[s].b] = (int)s;
    }
    for (size_t s = 0; s < p.steps.size(); ++s) {
        const StepPlan &st = p.steps[s];
        if (st.kblk) return *why = "K-blocked operands", false;
        SStep &S = P->step[s];
        S.mb = st.mb;
        S.nb = st.nb;
        S.kb = st.kb;
        if (st.mb + st.kb > 20 || st.nb + st.kb > 20 || st.mb + st.nb > 20) return *why = "step too large", false;
        S.a_src = st.a < p.m ? st.a : -1 - (st.a - p.m);
        S.b_src = st.b < p.m ? st.b : -1 - (st.b - p.m);
        if (st.maskR >> 32 || st.maskC >> 32) return *why = "result wider than 32 bits", false;
        S.maskR = (uint32_t)st.maskR;
        S.maskC = (uint32_t)st.maskC;
        const int64_t pk = pitch_of(1 << st.kb);
        if (S.a_src >= 0) stg[0] = std::max(stg[0], ((int64_t)1 << st.mb) * pk);
        if (S.b_src >= 0) stg[1] = std::max(stg[1], ((int64_t)1 << st.nb) * pk);
        const int M = 1 << st.mb, N = 1 << st.nb, K = 1 << st.kb;
        S.tm = std::min(4, M);
        S.tn = std::min(4, N);
        const int tiles = (M / S.tm) * (N / S.tn);
        int ks = 1;
        while (2 * ks * tiles <= ST_THREADS && K / (2 * ks) >= 4) ks *= 2;
        S.ksplit = ks;
        if (ks > 1) red = std::max(red, (int64_t)ks * M * N);
    }
    int64_t off = align4(stg[0]) + align4(stg[1]);
    P->red_off = (int32_t)off;
    off += align4(red);
    for (size_t s = 0; s < p.steps.size(); ++s) {
        SStep &S = P->step[s];
        const int c = consumer[(size_t)p.steps[s].c];
        if (c < 0) {  // the final step: a scalar per state
            if (S.mb != 0 || S.nb != 0) return *why = "final step is not a scalar", false;
            S.c_kb = -1;
            S.c_off = 0;
            continue;
        }
        S.c_kb = p.steps[(size_t)c].kb;
        S.c_off = (int32_t)off;
        const int64_t ck = (int64_t)1 << S.c_kb;
        off += align4((((int64_t)1 << (S.mb + S.nb)) / ck) * pitch_of((int)ck));
    }
    for (size_t s = 0; s < p.steps.size(); ++s) {
        SStep &S = P->step[s];
        S.a_off = S.a_src >= 0 ? 0 : P->step[-1 - S.a_src].c_off;
        S.b_off = S.b_src >= 0 ? (int32_t)align4(stg[0]) : P->step[-1 - S.b_src].c_off;
        S.tab_off = (int32_t)off;  // offset tables of the epilogue (ints)
        off += align4(((int64_t)1 << S.mb) + ((int64_t)1 << S.nb));
    }
    if (off > ST_MAX_SMEM_FLOATS) return *why = "intermediates exceed shared memory", false;
    P->smem_floats = (int32_t)std::max<int64_t>(off, 4);
    return true;
}

tqc_status cuda_fail(cudaError_t e, const char *what) {
    return fail(TQC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

// Shared-memory floats of the fused form, or -1 when the plan runs per state.
int states_fused_floats(const Plan &p) {
    SProgram P;
    std::string why;
    return build_program(p, &P, &why) ? P.smem_floats : -1;
}

tqc_status exec_contract_states(Plan *p, const uint64_t *states, int64_t n, void *d_out, int out_dtype,
                                double *z_out, void *stream) {
    if (!p->free_qubits.empty())
        return fail(TQC_ERR_INVALID, "state lists need a plan with no free qubits (use_free_mask = 1, masks 0)");
    if (p->n_slices() != 1) return fail(TQC_ERR_UNSUPPORTED, "state lists need an unsliced plan");
    if (p->net->n_qubits > 64) return fail(TQC_ERR_UNSUPPORTED, "state lists support up to 64 qubits");
    if (n < 0) return fail(TQC_ERR_INVALID, "negative state count");
    const uint64_t qmask = p->net->n_qubits == 64 ? ~0ull : ((1ull << p->net->n_qubits) - 1);
    for (int64_t i = 0; i < n; ++i)
        if (states[i] & ~qmask) return fail(TQC_ERR_INVALID, "state " + std::to_string(i) + " has bits beyond n_qubits");
    tqc_status st = exec_prepare(p);
    if (st != TQC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    ExecCtx c;
    c.ws = p->d_ws;
    c.zws = p->d_zws;
    c.zinfo = p->d_zinfo;
    c.kpart = p->d_kpart;
    if (p->z_version != p->net->version) {
        st = exec_total_mass(*p, c, stream);
        if (st != TQC_OK) return st;
        p->z_version = p->net->version;
    }
    SProgram P;
    std::string why;
    const bool fused = build_program(*p, &P, &why);
    const int esize = out_dtype == TQC_F64 ? 8 : 4;
    if (fused && n > 0) {
        // per-node tables Tt_j[x][cuts], rebuilt when the tensors changed
        if (p->tab_version != p->net->version || !p->d_tab) {
            int64_t need = 0;
            std::vector<int64_t> toff;
            for (int j = 0; j < p->m; ++j) {
                toff.push_back(need);
                need += ((p->net->nodes[j].elems * 4 + 255) / 256) * 256;
            }
            if (need > p->tab_bytes) {
                if (p->d_tab) cudaFree(p->d_tab);
                p->d_tab = nullptr;
                p->tab_bytes = 0;
                if (cudaMalloc(&p->d_tab, (size_t)need) != cudaSuccess) {
                    cudaGetLastError();
                    return fail(TQC_ERR_OOM, "state-list tables of " + std::to_string(need) + " bytes");
                }
                p->tab_bytes = need;
            }
            p->tab_off = toff;
            for (int j = 0; j < p->m; ++j) {
                const Node &nd = p->net->nodes[j];
                const TensorPlan &t = p->tensors[j];
                IngestArgs g;
                g.src = nd.d_data;
                g.src_dtype = nd.dtype;
                int b = 0;
                for (auto &md : t.layout.modes) {  // the leaf's own layout: its cut bits
                    const int pos = exec_src_pos_cut(nd, md.id);
                    g.srcpos[b++] = (int8_t)pos;
                    g.srcpos[b++] = (int8_t)(pos + 1);
                }
                for (size_t k = 0; k < nd.out_qubits.size(); ++k) g.srcpos[b++] = (int8_t)k;  // then x
                g.nbits = b;
                g.dst = (char *)p->d_tab + toff[(size_t)j];
                g.storage = ST_F32;
                cudaError_t e = launch_ingest(g, (int64_t)1 << b, s);
                if (e != cudaSuccess) return cuda_fail(e, "state-list table");
            }
            p->tab_version = p->net->version;
        }
        for (int j = 0; j < p->m; ++j) P.leaf[j].table = (const float *)((char *)p->d_tab + p->tab_off[(size_t)j]);
        if (n * 8 > p->states_bytes) {
            if (p->d_states) cudaFree(p->d_states);
            p->d_states = nullptr;
            p->states_bytes = 0;
            if (cudaMalloc(&p->d_states, (size_t)n * 8) != cudaSuccess) {
                cudaGetLastError();
                return fail(TQC_ERR_OOM, "state list of " + std::to_string(n) + " states");
            }
            p->states_bytes = n * 8;
        }
        cudaError_t e = cudaMemcpyAsync(p->d_states, states, (size_t)n * 8, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "state list upload");
        const size_t smem = (size_t)P.smem_floats * 4;
        static size_t attr = 0;
        if (smem > 48 * 1024 && smem > attr) {
            e = cudaFuncSetAttribute(states_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return cuda_fail(e, "state-list kernel attribute");
            attr = smem;
        }
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, states_kernel, ST_THREADS, smem);
        if (e != cudaSuccess || per_sm < 1) return fail(TQC_ERR_UNSUPPORTED, "state-list kernel does not fit an SM");
        const int64_t grid = std::min<int64_t>(n, (int64_t)per_sm * sm_count());
        states_kernel<<<(unsigned)grid, ST_THREADS, smem, s>>>(P, (const uint64_t *)p->d_states, n, d_out,
                                                              out_dtype == TQC_F64, p->d_zinfo);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "state-list kernel");
    } else if (n > 0) {
        // per state: the single-state plan with the state's bits as the fixed bits
        std::vector<uint8_t> fixed((size_t)p->net->n_qubits);
        c.compute_z = false;
        p->reuse_ok = false;  // the workspace now holds other states' intermediates
        for (int64_t i = 0; i < n; ++i) {
            for (int q = 0; q < p->net->n_qubits; ++q) fixed[(size_t)q] = (uint8_t)((states[i] >> q) & 1);
            st = exec_run(*p, c, fixed.data(), (char *)d_out + i * esize, out_dtype, stream, nullptr);
            if (st != TQC_OK) return st;
        }
    }
    if (z_out) {
        double zi[4];
        cudaError_t e = cudaMemcpyAsync(zi, p->d_zinfo, sizeof zi, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "z copy");
        *z_out = zi[0];
        if (((int *)(zi + 2))[0] != 0) {
            cudaMemsetAsync(p->d_zinfo + 2, 0, sizeof(int), s);
            return fail(TQC_ERR_TIMEOUT, "a tensor-core step gave up waiting on its pipeline");
        }
    }
    return TQC_OK;
}

}  // namespace tqc
