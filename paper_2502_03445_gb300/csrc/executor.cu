// Executor: workspace allocation and the launch sequence of a plan on the
// caller's stream.
//
//   for every slice (assignment of the sliced cut edges, §III-E-2):
//       ingest the leaves that depend on it (bin restriction + layout + cast)
//       run the pairwise steps; the last one expands the output indices into
//       the bin order and writes (or adds, in FP64, across slices)
//   total mass Z of the scalar network, scale = 2^{-|E|} / Z
//   FP64 slice sum -> output (when sliced)
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "launch.h"
#include "tqc_internal.h"

namespace tqc {

namespace {

tqc_status cuda_fail(cudaError_t e, const char *what) {
    return fail(TQC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define TQC_CUDA(call, what)                         \
    do {                                             \
        cudaError_t _e = (call);                     \
        if (_e != cudaSuccess) return cuda_fail(_e, what); \
    } while (0)

char *ws_ptr(void *base, int64_t off) { return (char *)base + off; }

// Source bit positions of a node tensor [c_0]..[c_{n-1}][x]: output qubit
// out_qubits[k] is bit k; cut axis d occupies bits n_out + 2(n_cut-1-d) (+1).
int src_pos_qubit(const Node &nd, int q) {
    for (size_t k = 0; k < nd.out_qubits.size(); ++k)
        if (nd.out_qubits[k] == q) return (int)k;
    return -1;
}
int src_pos_cut(const Node &nd, int c) {
    int n = (int)nd.cut_ids.size();
    for (int d = 0; d < n; ++d)
        if (nd.cut_ids[d] == c) return (int)nd.out_qubits.size() + 2 * (n - 1 - d);
    return -1;
}

// Ingest arguments of leaf j for slice `slice` (fixed output bits of the bin
// plus sliced cut values go to src_base).
IngestArgs leaf_args(const Plan &p, const TensorPlan &t, int j, const uint8_t *fixed, int64_t slice, bool zplan,
                     const ExecCtx *c = nullptr) {
    const Node &nd = p.net->nodes[j];
    IngestArgs g;
    const bool caller = c && c->node_data;
    g.src = caller ? c->node_data[j] : nd.d_data;
    g.src_dtype = caller ? c->node_dtype : nd.dtype;
    int64_t base = 0;
    if (!zplan) {
        std::vector<char> isfree(p.net->n_qubits, 0);
        for (int q : p.free_qubits) isfree[q] = 1;
        for (size_t k = 0; k < nd.out_qubits.size(); ++k) {
            int q = nd.out_qubits[k];
            if (!isfree[q] && fixed[q]) base += 1ll << k;
        }
    }
    for (size_t i = 0; i < p.sliced.size(); ++i) {
        int c = p.sliced[i];
        int pos = src_pos_cut(nd, c);
        if (pos < 0) continue;
        int64_t v = (slice >> (2 * i)) & 3;
        base += v << pos;
    }
    g.src_base = base;
    int b = 0;
    for (auto &md : t.layout.modes) {
        if (md.is_cut) {
            int pos = src_pos_cut(nd, md.id);
            g.srcpos[b++] = (int8_t)pos;
            g.srcpos[b++] = (int8_t)(pos + 1);
        } else {
            g.srcpos[b++] = (int8_t)src_pos_qubit(nd, md.id);
        }
    }
    g.nbits = b;
    // total mass: sum over every output bit (a node without outputs is a plain FP64 gather)
    g.reduce_bits = zplan ? (int)nd.out_qubits.size() : 0;
    if (zplan) g.storage = ST_F64;
    return g;
}

StepArgs step_args(const Plan &p, const std::vector<TensorPlan> &T, const StepPlan &st, void *ws, TileShape tile) {
    StepArgs a;
    const TensorPlan &ta = T[st.a], &tb = T[st.b];
    a.A = ws_ptr(ws, ta.offset);
    a.B = ws_ptr(ws, tb.offset);
    if (ta.storage == ST_BF16X2) a.A_lo = ws_ptr(ws, ta.offset + ta.plane_bytes);
    if (tb.storage == ST_BF16X2) a.B_lo = ws_ptr(ws, tb.offset + tb.plane_bytes);
    a.mb = st.mb;
    a.nb = st.nb;
    a.kb = st.kb;
    a.kblk = st.kblk ? 1 : 0;
    a.epi = make_epi(st.maskR, st.maskC, st.mb, st.nb, tile);
    (void)p;
    return a;
}

int epi_mode_of(int storage) {
    switch (storage) {
        case ST_BF16: return EPI_BF16;
        case ST_BF16X2: return EPI_BF16X2;
        case ST_TF32: return EPI_TF32;
        case ST_F64: return EPI_Z;
        default: return EPI_F32;
    }
}

tqc_status launch_step(const Plan &p, const StepPlan &st, StepArgs &a, int *d_err, cudaStream_t s) {
    cudaError_t e;
    if (st.klass == KC_UMMA) e = launch_umma_step(st.tile, st.prec, a, d_err, s);
    else e = launch_simt_step(st.tile, a, s);
    (void)p;
    if (e != cudaSuccess) return cuda_fail(e, "step launch");
    return TQC_OK;
}

TileShape tile_of(const StepPlan &st) {
    if (st.klass == KC_UMMA) return umma_tile(st.tile);
    return st.tile == SIMT_SMALLK ? smallk_tile(st.mb, st.nb, st.kb) : simt_tile(st.tile);
}

// ---------------------------------------------------------------- autotuner
// For every step, time each tile configuration that fits the step on the
// plan's own operands (CUDA events, best of three after one warm-up launch)
// and keep the fastest.  Results are cached process-wide by the step's
// shape and epilogue pattern, so equal steps of other plans reuse them.
struct TuneKey {
    int klass, prec, mb, nb, kb, mode, smallk;
    uint64_t maskR, maskC;
    bool operator<(const TuneKey &o) const {
        return std::tie(klass, prec, mb, nb, kb, mode, smallk, maskR, maskC) <
               std::tie(o.klass, o.prec, o.mb, o.nb, o.kb, o.mode, o.smallk, o.maskR, o.maskC);
    }
};
std::map<TuneKey, int> g_tune_cache;
std::mutex g_tune_mu;

std::vector<int> tile_candidates(const StepPlan &st, bool smallk) {
    std::vector<int> c;
    if (st.klass == KC_UMMA) {
        if (st.nb >= 7) c.push_back(UMMA_128x128);
        c.push_back(UMMA_128x64);
        if (st.mb >= 7 && st.nb >= 7) c.push_back(UMMA_128x128_DEEP);
        if (st.mb >= 7 && st.nb >= 8) c.push_back(UMMA_128x256_DEEP);
    } else {
        if (smallk && smallk_ok(st.mb, st.nb, st.kb, st.kblk)) c.push_back(SIMT_SMALLK);
        c.push_back(SIMT_64x64);
        if (st.mb >= 7 && st.nb >= 6) c.push_back(SIMT_128x64);
        if (st.mb >= 7 && st.nb >= 7) c.push_back(SIMT_128x128);
    }
    return c;
}

}  // namespace

namespace {

uint64_t host_pdep64(uint64_t src, uint64_t mask) {
    uint64_t r = 0;
    while (mask) {
        const uint64_t low = mask & (~mask + 1);
        if (src & 1) r |= low;
        src >>= 1;
        mask ^= low;
    }
    return r;
}

}  // namespace

// Fraction of the bytes of the 32-byte sectors that one warp store of the
// direct epilogue fills: lanes are 32 consecutive accumulator rows, each
// storing its run of vw consecutive elements (the rule of umma.cu).
double direct_store_efficiency(const EpiParams &e, int esize) {
    const int vw = ((e.lowCc & 3u) == 3u && e.L >= 2) ? 4 : ((e.lowCc & 1u) && e.L >= 1 ? 2 : 1);
    std::vector<uint64_t> sec;
    for (uint32_t r = 0; r < 32; ++r) {
        const uint64_t off = host_pdep64(host_pdep64(r, e.lowRc), e.tileMask);
        for (int i = 0; i < vw; ++i) sec.push_back((off + (uint64_t)i) * (uint64_t)esize >> 5);
    }
    std::sort(sec.begin(), sec.end());
    const size_t n = (size_t)(std::unique(sec.begin(), sec.end()) - sec.begin());
    return 32.0 * vw * esize / (32.0 * (double)n);
}

// Without autotuning: big tiles for big steps.  The direct-epilogue
// tensor-core form (*_DEEP) takes
//  * steps with a long K loop (K >= 2^12) over whole 128-row tiles: 128 x 256
//    tiles when N allows (1.3-1.5x over 128 x 128 at K = 2^14 in every
//    precision), 128 x 128 ones only for split BF16;
//  * steps whose direct warp stores fill whole 32-byte sectors (the result's
//    lowest bits are column bits, then row bits, as in the Kronecker
//    expansion of a final step), with 128 x 256 tiles when N allows (grid30's
//    final step: 0.92 ms against 1.50 ms staged), else 128 x 128 (grid30's
//    step 1, N = 128: 0.48 ms against 0.56 ms, the autotuner's choice).
// CUDA-core steps with K of 1, 4 or 16 take the small-K tile (unless
// `smallk` is false).
int default_step_tile(const StepPlan &st, int out_esize, bool smallk) {
    if (st.klass == KC_UMMA) {
        const bool big = st.mb >= 7 && st.nb >= 7;
        const bool deep = big && st.kb >= DEEP_MIN_LOG2_K;
        if (deep && st.nb >= 8) return UMMA_128x256_DEEP;
        if (deep) return st.prec == TQC_PREC_BF16X3 ? UMMA_128x128_DEEP : UMMA_128x128;
        if (big) {
            const EpiParams e = make_epi(st.maskR, st.maskC, st.mb, st.nb, TileShape{7, 6});
            if (direct_store_efficiency(e, out_esize) >= 0.99) return st.nb >= 8 ? UMMA_128x256_DEEP : UMMA_128x128_DEEP;
        }
        return st.nb >= 7 ? UMMA_128x128 : UMMA_128x64;
    }
    if (smallk && smallk_ok(st.mb, st.nb, st.kb, st.kblk)) return SIMT_SMALLK;
    return (st.mb >= 7 && st.nb >= 7) ? SIMT_128x128 : (st.mb >= 7 && st.nb >= 6 ? SIMT_128x64 : SIMT_64x64);
}

// K split of a final tensor-core step in the deep form.  T tiles on S SMs
// take ceil(T / S) waves of the whole K loop, so when T is not a multiple of
// S the last wave leaves SMs idle (512 tiles on 152 SMs: 3.37 waves take 4).
// Running k ranges of K as separate units evens the waves; each unit stores
// an FP32 partial and one reduce pass sums them in FP64.  Time model, in
// k-block units of about a microsecond: ceil(T k / S) (k_blocks / k + 4)
// (4 = pipeline fill and epilogue per unit), plus the reduce's bytes at HBM
// speed.  The smallest k within 2% of the best is taken, with at least 16
// k-blocks per range and the partials within max_part_bytes.
int step_ksplit(const StepPlan &st, int64_t out_elems, int64_t max_part_bytes) {
    if (!st.final || st.klass != KC_UMMA) return 1;
    if (st.tile != UMMA_128x128_DEEP && st.tile != UMMA_128x256_DEEP) return 1;
    const int lbn = st.tile == UMMA_128x256_DEEP ? 8 : 7;
    const int lbk = st.prec == TQC_PREC_TF32 ? 5 : 6;  // 128-byte k-blocks
    if (st.mb < 7 || st.nb < lbn || st.kb < lbk) return 1;
    const int64_t tiles = ((int64_t)1 << (st.mb - 7)) << (st.nb - lbn);
    const int64_t kblocks = (int64_t)1 << (st.kb - lbk);
    const int64_t sms = sm_count();
    constexpr int KMAX = 16;
    double cost[KMAX + 1];
    int kmax = 1;
    for (int k = 1; k <= KMAX; ++k) {
        if (k > 1 && (kblocks / k < 16 || (int64_t)k * out_elems * 4 > max_part_bytes)) break;
        const double waves = (double)((tiles * k + sms - 1) / sms);
        cost[k] = waves * ((double)kblocks / k + 4.0) * 1e-6 +
                  (k > 1 ? (4.0 * k + 16.0) * (double)out_elems / 6.8e12 + 5e-6 : 0.0);
        kmax = k;
    }
    double best = cost[1];
    for (int k = 2; k <= kmax; ++k) best = std::min(best, cost[k]);
    for (int k = 1; k <= kmax; ++k)
        if (cost[k] <= best * 1.02) return k;
    return 1;
}

// Sets every step's K split for its current tile and sizes the partials'
// buffer (allocated once, grown if the autotuner picked a tile that splits
// further).
tqc_status update_ksplit(Plan *p) {
    const int64_t cap = p->budget ? (int64_t)(p->budget / 16) : ((int64_t)1 << 30);
    int64_t need = 0;
    for (auto &st : p->steps) {
        st.ksplit = step_ksplit(st, p->out_elems(), cap);
        if (st.ksplit > 1) need = std::max(need, (int64_t)st.ksplit * p->out_elems() * 4);
    }
    if (need > p->kpart_bytes) {
        if (p->d_kpart) cudaFree(p->d_kpart);
        p->d_kpart = nullptr;
        p->kpart_bytes = 0;
        cudaError_t e = cudaMalloc(&p->d_kpart, (size_t)need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(TQC_ERR_OOM, "K-split partials of " + std::to_string(need) + " bytes");
        }
        p->kpart_bytes = need;
    }
    return TQC_OK;
}

int exec_src_pos_qubit(const Node &nd, int q) { return src_pos_qubit(nd, q); }
int exec_src_pos_cut(const Node &nd, int c) { return src_pos_cut(nd, c); }

IngestArgs exec_leaf_args(const Plan &p, const TensorPlan &t, int j, const uint8_t *fixed) {
    return leaf_args(p, t, j, fixed, 0, false);
}
StepArgs exec_step_args(const Plan &p, const StepPlan &st, TileShape tile) {
    return step_args(p, p.tensors, st, p.d_ws, tile);
}
int exec_epi_mode(int storage) { return epi_mode_of(storage); }

// Bytes per element the step's epilogue writes (a plane of a split-BF16
// operand counts 2; a final step 4, its FP64 forms store at least as wide).
int step_out_esize(const Plan &p, const StepPlan &st) {
    if (st.final) return 4;
    const int sg = p.tensors[st.c].storage;
    return (sg == ST_BF16 || sg == ST_BF16X2) ? 2 : (sg == ST_F64 ? 8 : 4);
}

tqc_status exec_autotune(Plan *p, void *d_out, int out_dtype, cudaStream_t s) {
    const bool sliced = p->n_slices() > 1;
    cudaEvent_t e0, e1;
    TQC_CUDA(cudaEventCreate(&e0), "event");
    TQC_CUDA(cudaEventCreate(&e1), "event");
    int *d_err = (int *)(p->d_zinfo + 2);
    tqc_status result = TQC_OK;
    for (StepPlan &sp : p->steps) {
        if (sp.fuse) continue;  // a fused pair has one configuration
        const TensorPlan &tc = p->tensors[sp.c];
        int mode = sp.final ? (sliced ? EPI_F64_SET : (out_dtype == TQC_F64 ? EPI_OUT_F64 : EPI_OUT_F32))
                            : epi_mode_of(tc.storage);
        const bool smallk = !(p->flags & TQC_FLAG_NO_SMALLK);
        TuneKey key{sp.klass, sp.prec, sp.mb, sp.nb, sp.kb, mode, smallk ? 1 : 0, sp.maskR, sp.maskC};
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) {
                sp.tile = it->second;
                continue;
            }
        }
        float best = 1e30f;
        int best_tile = sp.tile;
        for (int cand : tile_candidates(sp, smallk)) {
            StepPlan trial = sp;
            trial.tile = cand;
            StepArgs a = step_args(*p, p->tensors, trial, p->d_ws, tile_of(trial));
            a.epi.zinfo = p->d_zinfo;
            a.epi.mode = mode;
            if (sp.final) a.epi.out = sliced ? (out_dtype == TQC_F64 ? d_out : ws_ptr(p->d_ws, p->acc_offset)) : d_out;
            else {
                a.epi.out = ws_ptr(p->d_ws, tc.offset);
                if (tc.storage == ST_BF16X2) a.epi.out_lo = ws_ptr(p->d_ws, tc.offset + tc.plane_bytes);
            }
            float ms_min = 1e30f;
            for (int rep = 0; rep < 4 && result == TQC_OK; ++rep) {
                cudaEventRecord(e0, s);
                result = launch_step(*p, trial, a, d_err, s);
                cudaEventRecord(e1, s);
                if (result != TQC_OK) break;
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    result = fail(TQC_ERR_CUDA, "autotune timing");
                    break;
                }
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) ms_min = std::min(ms_min, ms);
            }
            if (result != TQC_OK) break;
            if (ms_min < best) {
                best = ms_min;
                best_tile = cand;
            }
        }
        if (result != TQC_OK) break;
        sp.tile = best_tile;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best_tile;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result == TQC_OK) {
        p->tuned = 1;
        result = update_ksplit(p);
    }
    return result;
}

// Allocates the plan's device state on its first contract.  A failure frees
// whatever this call allocated, so a later call starts again from nothing.
tqc_status exec_prepare(Plan *p) {
    if (p->ready) return TQC_OK;
    int dev = -1;
    TQC_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != p->net->device) return fail(TQC_ERR_INVALID, "current device differs from the network's device");
    auto oom = [&](const std::string &what) {
        cudaGetLastError();
        exec_release(p);
        return fail(TQC_ERR_OOM, what);
    };
    int64_t zslots = p->n_slices();
    if (p->ws_bytes > 0 && cudaMalloc(&p->d_ws, (size_t)p->ws_bytes) != cudaSuccess)
        return oom("workspace of " + std::to_string(p->ws_bytes) + " bytes");
    size_t zb = (size_t)p->zws_bytes + 8 * (size_t)zslots + 256;
    if (cudaMalloc(&p->d_zws, zb) != cudaSuccess) return oom("total-mass workspace");
    if (cudaMalloc((void **)&p->d_zinfo, 4 * sizeof(double) + 64) != cudaSuccess) return oom("zinfo");
    cudaError_t e = cudaMemset(p->d_zinfo, 0, 4 * sizeof(double) + 64);
    if (e != cudaSuccess) {
        exec_release(p);
        return cuda_fail(e, "memset");
    }
    // tile choice without autotuning: big tiles for big steps
    for (auto &st : p->steps) {
        st.tile = default_step_tile(st, step_out_esize(*p, st), !(p->flags & TQC_FLAG_NO_SMALLK));
    }
    tqc_status kst = update_ksplit(p);
    if (kst != TQC_OK) {
        exec_release(p);
        return kst;
    }
    p->ready = true;
    return TQC_OK;
}

void exec_clear_events(Plan *p) {
    for (auto &v : p->step_events)
        for (auto &pr : v) {
            cudaEventDestroy((cudaEvent_t)pr[0]);
            cudaEventDestroy((cudaEvent_t)pr[1]);
        }
    p->step_events.clear();
}

tqc_status exec_step_time(Plan *p, int step, double *mean_ms, int *launches) {
    double tot = 0;
    int n = 0;
    if (step < (int)p->step_events.size())
        for (auto &pr : p->step_events[step]) {
            TQC_CUDA(cudaEventSynchronize((cudaEvent_t)pr[1]), "event sync");
            float ms = 0;
            TQC_CUDA(cudaEventElapsedTime(&ms, (cudaEvent_t)pr[0], (cudaEvent_t)pr[1]), "event time");
            tot += ms;
            ++n;
        }
    if (mean_ms) *mean_ms = n ? tot / n : 0.0;
    if (launches) *launches = n;
    return TQC_OK;
}

void exec_release(Plan *p) {
    exec_clear_events(p);
    if (p->d_ws) cudaFree(p->d_ws);
    if (p->d_zws) cudaFree(p->d_zws);
    if (p->d_zinfo) cudaFree(p->d_zinfo);
    if (p->d_kpart) cudaFree(p->d_kpart);
    if (p->d_tab) cudaFree(p->d_tab);
    if (p->d_states) cudaFree(p->d_states);
    p->d_tab = p->d_states = nullptr;
    p->tab_bytes = p->states_bytes = 0;
    p->tab_version = 0;
    p->d_ws = p->d_zws = p->d_kpart = nullptr;
    p->kpart_bytes = 0;
    p->d_zinfo = nullptr;
    p->ready = false;
}

// Total mass Z of the network (every output summed: a scalar network per
// slice, FP64), then zinfo = [Z, scale = 2^{-|E|} / Z (or 2^{-|E|} without
// renormalisation)].
tqc_status exec_total_mass(const Plan &pl, const ExecCtx &c, void *stream) {
    const Plan *p = &pl;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t ns = p->n_slices();
    double *zslice = (double *)ws_ptr(c.zws, p->zws_bytes);
    for (int64_t sl = 0; sl < ns; ++sl) {
        for (int j = 0; j < p->m; ++j) {
            const TensorPlan &t = p->ztensors[j];
            IngestArgs g = leaf_args(*p, t, j, p->fixed_bits.data(), sl, true, &c);
            g.dst = p->m == 1 ? (void *)(zslice + sl) : (void *)ws_ptr(c.zws, t.offset);
            TQC_CUDA(launch_ingest(g, (int64_t)1 << t.nbits(), s), "total-mass ingest");
        }
        for (size_t i = 0; i < p->zsteps.size(); ++i) {
            const StepPlan &zs = p->zsteps[i];
            StepArgs a = step_args(*p, p->ztensors, zs, c.zws, simt_f64_tile());
            a.epi.mode = EPI_Z;
            a.epi.out = zs.final ? (void *)(zslice + sl) : (void *)ws_ptr(c.zws, p->ztensors[zs.c].offset);
            TQC_CUDA(launch_simt_step_f64(a, s), "total-mass step");
        }
    }
    TQC_CUDA(launch_zfinal(zslice, (int)ns, p->net->n_cuts, !(p->flags & TQC_FLAG_NO_RENORM), c.zinfo, s), "zfinal");
    return TQC_OK;
}

// The launch sequence of one contract.  Everything it reads and writes
// besides the caller's output comes from `c`.
tqc_status exec_run(Plan &pl, const ExecCtx &c, const uint8_t *fixed_bits, void *d_out, int out_dtype, void *stream,
                    bool *z_computed, const std::vector<char> *keep) {
    Plan *p = &pl;
    cudaStream_t s = (cudaStream_t)stream;
    tqc_status st = TQC_OK;
    if (z_computed) *z_computed = false;
    const uint8_t *fixed = fixed_bits ? fixed_bits : p->fixed_bits.data();
    if (fixed_bits)
        for (int q = 0; q < p->net->n_qubits; ++q)
            if (fixed_bits[q] > 1) return fail(TQC_ERR_INVALID, "fixed_bits entries must be 0 or 1");
    const int64_t ns = p->n_slices();
    // a step's tile: the plan's (autotuned or default), or the default and unsplit
    auto step_of = [&](const StepPlan &sp) {
        StepPlan x = sp;
        if (c.default_tiles) {
            x.tile = default_step_tile(sp, step_out_esize(*p, sp), !(p->flags & TQC_FLAG_NO_SMALLK));
            x.ksplit = 1;
        }
        return x;
    };

    // ---- total mass Z (scalar network: every output summed), FP64.  Z depends
    // on the tensors only, so the allocating path recomputes it only when they
    // changed since the plan last computed it.
    if (c.compute_z) {
        st = exec_total_mass(*p, c, stream);
        if (st != TQC_OK) return st;
        if (z_computed) *z_computed = true;
    }

    // ---- single subcircuit: the bin is a gather of its tensor
    if (p->m == 1) {
        const TensorPlan &t = p->tensors[0];
        IngestArgs g = leaf_args(*p, t, 0, fixed, 0, false, &c);
        g.dst = d_out;
        g.scaled = 1;
        g.out_f64 = out_dtype == TQC_F64;
        g.zinfo = c.zinfo;
        TQC_CUDA(launch_ingest(g, p->out_elems(), s), "ingest");
        return TQC_OK;
    }
    const bool sliced = ns > 1;
    double *acc = nullptr;
    if (sliced) acc = out_dtype == TQC_F64 ? (double *)d_out : (double *)ws_ptr(c.ws, p->acc_offset);
    int *d_err = (int *)(c.zinfo + 2);
    for (int64_t sl = 0; sl < ns; ++sl) {
        for (int j = 0; j < p->m; ++j) {
            const TensorPlan &t = p->tensors[j];
            if (sl > 0 && !t.slice_dep) continue;
            if (keep && (*keep)[(size_t)j]) continue;  // still in the workspace from the last call
            IngestArgs g = leaf_args(*p, t, j, fixed, sl, false, &c);
            g.dst = ws_ptr(c.ws, t.offset);
            if (t.storage == ST_BF16X2) g.dst_lo = ws_ptr(c.ws, t.offset + t.plane_bytes);
            g.storage = t.storage;
            TQC_CUDA(launch_ingest(g, (int64_t)1 << t.nbits(), s), "ingest");
        }
        for (size_t si = 0; si < p->steps.size(); ++si) {
            const StepPlan sp = step_of(p->steps[si]);
            if (sp.fuse == 2) continue;  // ran inside the previous step's fused kernel
            if (sl > 0 && !p->tensors[sp.c].slice_dep) continue;
            if (sp.fuse == 1) {
                // steps si and si + 1 as one kernel: the intermediate stays on chip
                const StepPlan sp1 = step_of(p->steps[si + 1]);
                if (keep && (*keep)[(size_t)sp1.c]) continue;
                StepArgs a0 = step_args(*p, p->tensors, sp, c.ws, TileShape{7, 6});
                StepArgs a1 = step_args(*p, p->tensors, sp1, c.ws, TileShape{7, 6});
                const TensorPlan &t1 = p->tensors[sp1.c];
                a1.epi.zinfo = c.zinfo;
                a1.epi.out = ws_ptr(c.ws, t1.offset);
                if (t1.storage == ST_BF16X2) a1.epi.out_lo = ws_ptr(c.ws, t1.offset + t1.plane_bytes);
                a1.epi.mode = epi_mode_of(t1.storage);
                cudaEvent_t ev[2] = {nullptr, nullptr};
                if (c.profile) {
                    TQC_CUDA(cudaEventCreate(&ev[0]), "event");
                    TQC_CUDA(cudaEventCreate(&ev[1]), "event");
                    TQC_CUDA(cudaEventRecord(ev[0], s), "event record");
                }
                TQC_CUDA(launch_fused_pair(a0, a1, sp.maskR, sp.maskC, d_err, s), "fused step launch");
                if (c.profile) {
                    TQC_CUDA(cudaEventRecord(ev[1], s), "event record");
                    if (p->step_events.size() < p->steps.size()) p->step_events.resize(p->steps.size());
                    p->step_events[si].push_back({(void *)ev[0], (void *)ev[1]});
                }
                continue;
            }
            if (keep && (*keep)[(size_t)sp.c]) continue;
            StepArgs a = step_args(*p, p->tensors, sp, c.ws, tile_of(sp));
            const TensorPlan &tc = p->tensors[sp.c];
            a.epi.zinfo = c.zinfo;
            if (sp.final) {
                if (sliced) {
                    a.epi.out = acc;
                    a.epi.mode = sl == 0 ? EPI_F64_SET : EPI_F64_ADD;
                } else {
                    a.epi.out = d_out;
                    a.epi.mode = out_dtype == TQC_F64 ? EPI_OUT_F64 : EPI_OUT_F32;
                }
            } else {
                a.epi.out = ws_ptr(c.ws, tc.offset);
                if (tc.storage == ST_BF16X2) a.epi.out_lo = ws_ptr(c.ws, tc.offset + tc.plane_bytes);
                a.epi.mode = epi_mode_of(tc.storage);
            }
            cudaEvent_t ev[2] = {nullptr, nullptr};
            if (c.profile) {
                TQC_CUDA(cudaEventCreate(&ev[0]), "event");
                TQC_CUDA(cudaEventCreate(&ev[1]), "event");
                TQC_CUDA(cudaEventRecord(ev[0], s), "event record");
            }
            if (sp.ksplit > 1) {
                // split K: FP32 partials, then one pass into the step's own output mode
                void *out = a.epi.out;
                const int mode = a.epi.mode;
                a.ksplit = sp.ksplit;
                a.split_stride = p->out_elems();
                a.epi.out = c.kpart;
                a.epi.mode = EPI_F32;
                st = launch_step(*p, sp, a, d_err, s);
                if (st != TQC_OK) return st;
                TQC_CUDA(launch_ksplit_reduce((const float *)c.kpart, sp.ksplit, p->out_elems(), mode, out, c.zinfo,
                                              s),
                         "K-split reduce");
            } else {
                st = launch_step(*p, sp, a, d_err, s);
                if (st != TQC_OK) return st;
            }
            if (c.profile) {
                TQC_CUDA(cudaEventRecord(ev[1], s), "event record");
                if (p->step_events.size() < p->steps.size()) p->step_events.resize(p->steps.size());
                p->step_events[si].push_back({(void *)ev[0], (void *)ev[1]});
            }
        }
    }
    if (sliced) TQC_CUDA(launch_finalize(acc, d_out, out_dtype == TQC_F64, c.zinfo, p->out_elems(), s), "finalize");
    return TQC_OK;
}

tqc_status exec_contract(Plan *p, const uint8_t *fixed_bits, void *d_out, int out_dtype, double *z_out,
                         void *stream) {
    tqc_status st = exec_prepare(p);
    if (st != TQC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (p->autotune && !p->tuned) {
        st = exec_autotune(p, d_out, out_dtype, s);
        if (st != TQC_OK) return st;
    }
    ExecCtx c;
    c.ws = p->d_ws;
    c.zws = p->d_zws;
    c.zinfo = p->d_zinfo;
    c.kpart = p->d_kpart;
    c.compute_z = p->z_version != p->net->version;
    c.profile = p->profile != 0;
    if (fixed_bits)
        for (int q = 0; q < p->net->n_qubits; ++q)
            if (fixed_bits[q] > 1) return fail(TQC_ERR_INVALID, "fixed_bits entries must be 0 or 1");
    // Tensors whose leaves all kept their bin restriction since the last call
    // (same tensor version) are still valid in the workspace; slice-dependent
    // ones were overwritten by later slices, and the root is the output.
    const uint8_t *fixed = fixed_bits ? fixed_bits : p->fixed_bits.data();
    std::vector<int64_t> keys((size_t)p->m);
    for (int j = 0; j < p->m; ++j) keys[(size_t)j] = leaf_args(*p, p->tensors[(size_t)j], j, fixed, 0, false).src_base;
    std::vector<char> keep(p->tensors.size(), 0);
    p->reused_leaves = p->reused_steps = 0;
    if ((p->flags & TQC_FLAG_REUSE) && !p->batched && p->reuse_ok && p->reuse_version == p->net->version &&
        p->m > 1) {
        uint64_t dirty = 0;
        for (int j = 0; j < p->m; ++j)
            if (keys[(size_t)j] != p->leaf_key[(size_t)j]) dirty |= 1ull << j;
        for (size_t i = 0; i + 1 < p->tensors.size(); ++i) {
            const TensorPlan &t = p->tensors[i];
            if (t.slice_dep || (t.leaves & dirty)) continue;
            keep[i] = 1;
            if ((int)i < p->m) ++p->reused_leaves;
            else ++p->reused_steps;
        }
    }
    p->reuse_ok = false;  // set again once every launch of this call is issued
    bool zc = false;
    st = exec_run(*p, c, fixed_bits, d_out, out_dtype, stream, &zc, &keep);
    if (st != TQC_OK) return st;
    if (zc) p->z_version = p->net->version;
    p->leaf_key = keys;
    p->reuse_version = p->net->version;
    p->reuse_ok = true;
    if (z_out) {
        // Z, the scale and the error word, which stays set from the call whose
        // bounded wait gave up until a call with z_out reports (and clears) it
        double zi[4];
        TQC_CUDA(cudaMemcpyAsync(zi, p->d_zinfo, sizeof zi, cudaMemcpyDeviceToHost, s), "z copy");
        TQC_CUDA(cudaStreamSynchronize(s), "sync");
        *z_out = zi[0];
        if (((int *)(zi + 2))[0] != 0) {
            TQC_CUDA(cudaMemsetAsync(p->d_zinfo + 2, 0, sizeof(int), s), "error word clear");
            return fail(TQC_ERR_TIMEOUT, "a tensor-core step gave up waiting on its pipeline");
        }
    }
    return TQC_OK;
}

// The steps first..end of a plan whose leaf operands and earlier results
// are already in its workspace (the batched launch's large steps), launched
// as tqc_contract would launch them, with the plan's cached total mass.
tqc_status exec_run_tail(Plan &p, size_t first, void *d_out, void *stream) {
    ExecCtx c;
    c.ws = p.d_ws;
    c.zws = p.d_zws;
    c.zinfo = p.d_zinfo;
    c.kpart = p.d_kpart;
    std::vector<char> keep(p.tensors.size(), 0);
    for (int j = 0; j < p.m; ++j) keep[(size_t)j] = 1;
    for (size_t i = 0; i < first && i < p.steps.size(); ++i) keep[(size_t)p.steps[i].c] = 1;
    return exec_run(p, c, nullptr, d_out, TQC_F32, stream, nullptr, &keep);
}

}  // namespace tqc
