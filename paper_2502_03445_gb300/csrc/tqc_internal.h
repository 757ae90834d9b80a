// Internal data structures of libtqc: network IR, plan IR and the launch
// parameter blocks shared by the host executor and the kernels.
#pragma once

#include <array>
#include <cstdint>
#include <string>
#include <vector>

#include "tqc.h"

struct tqc_costmodel;

namespace tqc {

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
tqc_status fail(tqc_status st, const std::string &msg);

// ---------------------------------------------------------------- network
struct Node {
    std::vector<int> out_qubits;  // bit k of x = out_qubits[k]
    std::vector<int> cut_ids;     // axis d = cut_ids[d]
    std::vector<int8_t> cut_role; // 0 upstream, 1 downstream
    int dtype = TQC_F64;          // dtype of the device copy
    void *d_data = nullptr;
    int64_t elems = 0;
};

struct Net {
    int n_qubits = 0;
    int n_cuts = 0;
    std::vector<Node> nodes;
    std::vector<std::array<int, 2>> cut_nodes;  // cut -> {upstream node, downstream node}
    bool has_data = false;
    int device = 0;
    int live_plans = 0;
    uint64_t version = 1;  // bumped whenever tensor data changes
};

// ---------------------------------------------------------------- layouts
// A tensor index is a bit string; every mode is a bit field: an output
// qubit (1 bit) or a cut edge (2 bits, value 0..3 = I,X,Y,Z, low bit first).
struct Mode {
    int8_t is_cut;
    int16_t id;
    int bits() const { return is_cut ? 2 : 1; }
    bool operator==(const Mode &o) const { return is_cut == o.is_cut && id == o.id; }
};

struct Layout {
    std::vector<Mode> modes;  // least significant first
    int nbits() const {
        int n = 0;
        for (auto &m : modes) n += m.bits();
        return n;
    }
    // bit position of the lowest bit of mode `m`, or -1
    int pos(const Mode &m) const {
        int p = 0;
        for (auto &x : modes) {
            if (x == m) return p;
            p += x.bits();
        }
        return -1;
    }
};

enum Storage { ST_F32 = 0, ST_BF16 = 1, ST_BF16X2 = 2, ST_F64 = 3, ST_TF32 = 4 };

inline int storage_bytes(int st) {
    switch (st) {
        case ST_BF16: return 2;
        case ST_BF16X2: return 4;  // two planes of 2 bytes
        case ST_F64: return 8;
        default: return 4;
    }
}

enum KernelClass { KC_SIMT = 0, KC_UMMA = 1 };

struct TensorPlan {
    uint64_t leaves = 0;          // leaf set (bit j = node j)
    std::vector<int> qubits;      // free output qubits, ascending
    std::vector<int> cuts;        // open cut edges (not sliced, not yet contracted), ascending
    Layout layout;
    int storage = ST_F32;
    int64_t offset = 0;           // workspace byte offset (plane 0)
    int64_t plane_bytes = 0;      // bytes of one plane
    bool slice_dep = false;       // depends on a sliced cut
    int nbits() const { return (int)qubits.size() + 2 * (int)cuts.size(); }
};

struct StepPlan {
    int a = -1, b = -1, c = -1;   // tensor ids: a = rows (M), b = cols (N), c = result
    int mb = 0, nb = 0, kb = 0;   // log2 of M, N, K
    int klass = KC_SIMT;
    int prec = TQC_PREC_FP32;
    uint64_t maskR = 0, maskC = 0;  // result-layout bits of row / column index bits
    bool final = false;
    int tile = 0;                 // tile configuration (autotuner)
    int ksplit = 1;               // K ranges run by separate CTAs (final tensor-core steps with few tiles)
    bool kblk = false;            // operands stored K-blocked: [K / 64][rows][64] (tensor-core steps with long rows)
    int fuse = 0;                 // 1: runs with the next step as one fused kernel; 2: run by the previous step's
};

// ---------------------------------------------------------------- cost model
struct CostConsts {
    double hbm_Bps = 6.79e12;       // measured copy bandwidth of this part
    double simt_fps = 5.0e13;       // sustained FP32 CUDA-core rate of the plain step kernel
    double bf16_fps = 1.6e15;       // sustained BF16 tcgen05 rate
    double tf32_fps = 0.65e15;      // measured on 128 x 256 tiles at K = 2^10 (655-667 TF/s)
    double launch_s = 3.0e-6;       // per kernel launch / tail
};

struct StepCost {
    double macs = 0, bytes = 0, time_s = 0;
};

// ---------------------------------------------------------------- plan
struct Plan {
    Net *net = nullptr;
    int m = 0;
    std::vector<int> free_qubits;          // ascending
    std::vector<uint8_t> fixed_bits;       // n_qubits
    int precision = TQC_PREC_FP32;
    int planner = TQC_PLANNER_GREEDY;
    std::string planner_used;              // how the order was chosen
    int flags = 0;
    int autotune = 0;
    uint64_t budget = 0;
    std::vector<std::array<int, 2>> order; // SSA pairs
    std::vector<int> sliced;               // sliced cuts, ascending
    std::vector<TensorPlan> tensors;       // leaves 0..m-1, step results m..
    std::vector<StepPlan> steps;
    std::vector<TensorPlan> ztensors;      // scalar network for Z (no outputs, no slicing)
    std::vector<StepPlan> zsteps;
    double flops = 0, bytes = 0, predicted_s = 0;
    int64_t ws_bytes = 0;                  // main workspace bytes
    int64_t zws_bytes = 0;
    int64_t acc_offset = -1;               // FP64 slice accumulator (when sliced and out is F32)
    std::string describe_json;
    // ---- device state (executor)
    void *d_ws = nullptr;
    void *d_zws = nullptr;
    double *d_zinfo = nullptr;             // [Z, scale]
    void *d_kpart = nullptr;               // FP32 partials of K-split steps
    int64_t kpart_bytes = 0;
    void *d_hostout = nullptr;             // buffer for tqc_contract_host
    int64_t d_hostout_bytes = 0;
    bool ready = false;
    int tuned = 0;
    int profile = 0;
    uint64_t z_version = 0;                // network version the cached Z belongs to
    void *d_tab = nullptr;                 // state lists: per-node tables Tt_j[x][cuts] (FP32)
    int64_t tab_bytes = 0;
    std::vector<int64_t> tab_off;
    uint64_t tab_version = 0;              // network version the tables belong to
    void *d_states = nullptr;              // state lists: the last list, on the device
    int64_t states_bytes = 0;
    // intermediates kept across calls (bins that differ in some leaves' fixed bits)
    bool reuse_ok = false;                 // the workspace holds the last call's values
    bool batched = false;                  // part of a batched launch, whose replays rewrite the workspace
    uint64_t reuse_version = 0;            // network version of those values
    std::vector<int64_t> leaf_key;         // per leaf: its bin restriction (source offset) in that call
    int reused_leaves = 0, reused_steps = 0;  // skipped in the last call
    std::vector<std::vector<std::array<void *, 2>>> step_events;  // per step: (start, stop) cudaEvent_t
    int64_t n_slices() const { return (int64_t)1 << (2 * sliced.size()); }
    int64_t out_elems() const { return (int64_t)1 << free_qubits.size(); }
};

// planner entry points (planner.cpp)
tqc_status build_plan(Net *net, const tqc_plan_opts &opts, Plan *plan);
std::string plan_describe(const Plan &p);
std::vector<std::vector<int32_t>> plan_candidate_orders(Net *net, const tqc_plan_opts &o, int max_n);

// learned cost model (costmodel.cu)
constexpr int kPlanFeatures = 32;
tqc_status costmodel_for_path(const char *path, ::tqc_costmodel **out);
tqc_status costmodel_predict_host(::tqc_costmodel *cm, const float *h_X, int n, float *h_y);
int costmodel_n_in(::tqc_costmodel *cm);
StepCost step_cost(int mb, int nb, int kb, int klass, int prec, const CostConsts &cc);
std::vector<double> plan_features(const Plan &p);   // learned cost-model features
int choose_class(int mb, int nb, int kb, int prec);
int step_prec(int prec, int mb, int nb, int kb);  // per-step operand type (resolves TQC_PREC_AUTO)

// Where one contract reads and writes.  The allocating path uses the
// plan's own device state; the allocation-free entry point points every
// buffer at its fixed scratch array and reads the caller's tensors, so it
// never touches the plan's or the network's device state.
struct ExecCtx {
    void *ws = nullptr;                      // main workspace
    void *zws = nullptr;                     // total-mass network (per-slice masses follow it)
    double *zinfo = nullptr;                 // [Z, scale, error word]
    void *kpart = nullptr;                   // FP32 partials of K-split steps
    const void *const *node_data = nullptr;  // per subcircuit; NULL = the network's device copies
    int node_dtype = TQC_F64;                // element type of node_data
    bool default_tiles = false;              // default tile of every step and no K split
    bool compute_z = false;                  // compute the total mass (else only when stale)
    bool profile = false;                    // record per-step events in the plan
};

// executor entry points (executor.cu)
tqc_status exec_prepare(Plan *p);
// The launch sequence of one contract on `stream` (no allocation, no
// synchronisation).  *z_computed tells whether the total mass was computed.
tqc_status exec_run(Plan &p, const ExecCtx &c, const uint8_t *fixed_bits, void *d_out, int out_dtype,
                    void *stream, bool *z_computed, const std::vector<char> *keep = nullptr);
// Steps first..end of an unsliced plan whose leaves and earlier step results
// are already in its workspace, FP32 output (the batched launch's tail).
tqc_status exec_run_tail(Plan &p, size_t first, void *d_out, void *stream);
// Arbitrary state list (states.cu): P(x) of n states on a plan with no free qubits.
tqc_status exec_contract_states(Plan *p, const uint64_t *states, int64_t n, void *d_out, int out_dtype,
                                double *z_out, void *stream);
// Shared-memory floats of the fused state-list kernel for a plan, or -1 when
// the plan's states run one at a time through the ordinary step kernels.
int states_fused_floats(const Plan &p);
// Total mass Z into c.zinfo (and the output scale), stream-ordered.
tqc_status exec_total_mass(const Plan &p, const ExecCtx &c, void *stream);
// Device source bit positions of a node tensor: output qubit q, cut c (-1 if absent).
int exec_src_pos_qubit(const Node &nd, int q);
int exec_src_pos_cut(const Node &nd, int c);
tqc_status exec_contract(Plan *p, const uint8_t *fixed_bits, void *d_out, int out_dtype, double *z_out,
                         void *stream);
void exec_release(Plan *p);
void exec_clear_events(Plan *p);
tqc_status exec_step_time(Plan *p, int step, double *mean_ms, int *launches);

// ---------------------------------------------------------------- launch blocks
// Epilogue of a pairwise step: where element (r, c) of the GEMM result goes.
// out offset = pdep(r_tile, highR) | pdep(c_tile, highC) | pdep(t, tileMask)
// with t = pdep(i, lowRc) | pdep(j, lowCc) for the tile-local row i, column j.
enum EpiMode {
    EPI_F32 = 0,        // operand for a CUDA-core step
    EPI_BF16 = 1,       // operand for a BF16 tensor-core step
    EPI_BF16X2 = 2,     // hi plane + lo plane (split BF16)
    EPI_TF32 = 3,       // FP32 rounded to TF32
    EPI_F64_SET = 4,    // first slice of the FP64 slice sum
    EPI_F64_ADD = 5,    // further slices
    EPI_OUT_F32 = 6,    // final output, scaled
    EPI_OUT_F64 = 7,    // final output, scaled, FP64
    EPI_Z = 8           // scalar-network step (FP64, unscaled)
};

struct EpiParams {
    void *out = nullptr;
    void *out_lo = nullptr;        // lo plane for EPI_BF16X2
    const double *zinfo = nullptr; // device [Z, scale]
    uint64_t highR = 0, highC = 0;
    uint64_t tileMask = 0;
    uint32_t lowRc = 0, lowCc = 0;
    int32_t a_bits = 0, b_bits = 0;  // tile-local row / column bits
    int32_t L = 0;                   // trailing ones of tileMask
    int32_t mode = EPI_F32;
};

struct StepArgs {
    const void *A = nullptr, *B = nullptr;
    const void *A_lo = nullptr, *B_lo = nullptr;
    int32_t mb = 0, nb = 0, kb = 0;
    EpiParams epi;
    // K split: split s of ksplit covers k-blocks [s kB / ksplit, (s+1) kB / ksplit)
    // and stores its FP32 partial (EPI_F32) at epi.out + s * split_stride
    int32_t ksplit = 1;
    int64_t split_stride = 0;
    // operands K-blocked: element (r, k) at (k / 64) * rows * 64 + r * 64 + k % 64
    int32_t kblk = 0;
};

struct IngestArgs {
    const void *src = nullptr;
    int32_t src_dtype = TQC_F64;
    int64_t src_base = 0;        // element offset of fixed bits and sliced cut values
    int32_t nbits = 0;           // destination bits
    int8_t srcpos[64] = {0};     // source bit position of each destination bit
    void *dst = nullptr;
    void *dst_lo = nullptr;
    int32_t storage = ST_F32;    // or the EPI_OUT_* scaled forms via `scaled`
    int32_t scaled = 0;          // multiply by zinfo[1] (single-node networks)
    int32_t out_f64 = 0;
    const double *zinfo = nullptr;
    int32_t reduce_bits = 0;     // > 0: sum over the 2^reduce_bits low source elements (Z)
};

}  // namespace tqc
