// Contraction planner: order search (§III-E-1), two-tier slicing (§III-E-2),
// per-step kernel class and precision, and the bit-field layouts of every
// operand and intermediate.
//
// Cost unit.  A pairwise step C[a,b] = sum_k A[a,k] B[k,b] costs
// dim(a)*dim(k)*dim(b) multiplications (§III-B, Fig. tensor_contraction); per
// reconstructed state that is 4^{#cuts of the step} (§III-C, Eq.
// tn_upper_bound).  Here a step's rows a are the left operand's free output
// qubits and open cuts that are not shared, its columns b the right ones, and
// k the shared cuts, so with F free qubits in the bin the multiply-adds of a
// step are 2^{log2 M + log2 N + log2 K}.  The predicted time of a step is the
// larger of its arithmetic at the rate of its kernel class and its algorithmic
// HBM bytes at the measured bandwidth, plus a launch cost.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <limits>
#include <sstream>

#include "launch.h"
#include "tqc_internal.h"

namespace tqc {

namespace {

inline int popc(uint64_t x) { return __builtin_popcountll(x); }

struct NetBits {
    int m = 0;
    std::vector<int> nfree;        // free output qubits per node
    std::vector<uint64_t> cutmask; // cut edges per node
    uint64_t sliced = 0;
};

NetBits net_bits(const Plan &p) {
    NetBits nb;
    nb.m = p.m;
    std::vector<char> isfree(p.net->n_qubits, 0);
    for (int q : p.free_qubits) isfree[q] = 1;
    for (auto &nd : p.net->nodes) {
        int f = 0;
        for (int q : nd.out_qubits) f += isfree[q];
        nb.nfree.push_back(f);
        uint64_t cm = 0;
        for (int c : nd.cut_ids) cm |= 1ull << c;
        nb.cutmask.push_back(cm);
    }
    for (int c : p.sliced) nb.sliced |= 1ull << c;
    return nb;
}

struct SubsetInfo {
    int q = 0;          // free qubits
    uint64_t cuts = 0;  // open cuts (unsliced)
};

SubsetInfo subset_info(const NetBits &nb, uint64_t leaves) {
    SubsetInfo s;
    uint64_t cm = 0;
    for (int j = 0; j < nb.m; ++j)
        if (leaves >> j & 1) {
            s.q += nb.nfree[j];
            cm ^= nb.cutmask[j];
        }
    s.cuts = cm & ~nb.sliced;
    return s;
}

struct StepShape {
    int mb, nb, kb;
};

StepShape pair_shape(const SubsetInfo &x, const SubsetInfo &y) {
    uint64_t shared = x.cuts & y.cuts;
    StepShape s;
    s.mb = x.q + 2 * popc(x.cuts & ~shared);
    s.nb = y.q + 2 * popc(y.cuts & ~shared);
    s.kb = 2 * popc(shared);
    if (s.mb < s.nb) std::swap(s.mb, s.nb);
    return s;
}

int in_bytes_of(int klass, int prec) {
    if (klass == KC_SIMT) return 4;
    if (prec == TQC_PREC_BF16) return 2;
    return 4;  // TF32 (FP32 storage) or BF16X3 (two BF16 planes)
}

}  // namespace

// Operand type of one tensor-core step.  A given precision applies to every
// step; under TQC_PREC_AUTO each step takes TF32 when split BF16 would leave
// it bound by the tensor pipe (its three MMAs per product take longer than
// moving its algorithmic HBM bytes), where TF32's single MMA per product at
// half the BF16 rate is 1.5x faster; every other step keeps split BF16: an
// HBM-bound step gains nothing from TF32 (both store 4 bytes per element)
// and split BF16 is the more accurate (operands exact to about 2^-16
// relative, against 2^-11 for TF32).
int step_prec(int prec, int mb, int nb, int kb) {
    if (prec != TQC_PREC_AUTO) return prec;
    const CostConsts cc;
    const double macs = std::ldexp(1.0, mb + nb + kb);
    const double bytes = 4.0 * (std::ldexp(1.0, mb + kb) + std::ldexp(1.0, nb + kb)) + 4.0 * std::ldexp(1.0, mb + nb);
    const double t_split_bf16 = 2.0 * macs * 3.0 / cc.bf16_fps;
    return t_split_bf16 > bytes / cc.hbm_Bps ? TQC_PREC_TF32 : TQC_PREC_BF16X3;
}

int choose_class(int mb, int nb, int kb, int prec) {
    if (prec == TQC_PREC_FP32) return KC_SIMT;
    // tensor cores only where the step is a real contraction: K >= 64 and a
    // result of at least one 128 x 128 tile
    if (kb >= 6 && mb + nb >= 14 && mb >= 4 && nb >= 4) return KC_UMMA;
    return KC_SIMT;
}

StepCost step_cost(int mb, int nb, int kb, int klass, int prec, const CostConsts &cc) {
    StepCost c;
    prec = step_prec(prec, mb, nb, kb);
    c.macs = std::ldexp(1.0, mb + nb + kb);
    int ib = in_bytes_of(klass, prec);
    c.bytes = ib * (std::ldexp(1.0, mb + kb) + std::ldexp(1.0, nb + kb)) + 4.0 * std::ldexp(1.0, mb + nb);
    double rate = cc.simt_fps;
    if (klass == KC_UMMA) {
        rate = prec == TQC_PREC_TF32 ? cc.tf32_fps : cc.bf16_fps;
        if (prec == TQC_PREC_BF16X3) rate /= 3.0;
        // a step narrower than one MMA tile wastes the rest of it
        if (mb < 7) rate *= std::ldexp(1.0, mb - 7);
    }
    c.time_s = std::max(2.0 * c.macs / rate, c.bytes / cc.hbm_Bps) + cc.launch_s;
    return c;
}

namespace {

// The plan-level precision: TQC_PREC_AUTO stays AUTO and is resolved per
// step by step_prec.
int effective_prec(int prec) { return prec; }

// Step cost under one of three objectives: 0 = predicted time (default),
// 1 = multiply-adds only (the paper's cost unit), 2 = HBM bytes only.
thread_local int g_cost_mode = 0;

double pair_time(const NetBits &nb, uint64_t x, uint64_t y, int prec, const CostConsts &cc) {
    StepShape s = pair_shape(subset_info(nb, x), subset_info(nb, y));
    int k = choose_class(s.mb, s.nb, s.kb, prec);
    StepCost c = step_cost(s.mb, s.nb, s.kb, k, prec, cc);
    return g_cost_mode == 1 ? c.macs : g_cost_mode == 2 ? c.bytes : c.time_s;
}

// Optimal tree for the additive step-cost model by dynamic programming over
// leaf subsets (every binary tree is reachable; 3^m work).
std::vector<std::array<uint64_t, 2>> exhaustive_tree(const NetBits &nb, int prec, const CostConsts &cc) {
    int m = nb.m;
    uint64_t full = (m == 64) ? ~0ull : ((1ull << m) - 1);
    std::vector<double> best(1ull << m, std::numeric_limits<double>::infinity());
    std::vector<uint64_t> split(1ull << m, 0);
    for (int j = 0; j < m; ++j) best[1ull << j] = 0.0;
    for (uint64_t S = 1; S <= full; ++S) {
        if (popc(S) < 2) continue;
        uint64_t low = S & (~S + 1);  // keep the lowest leaf in S1 to halve the work
        for (uint64_t S1 = (S - 1) & S; S1; S1 = (S1 - 1) & S) {
            if (!(S1 & low)) continue;
            uint64_t S2 = S ^ S1;
            double c = best[S1] + best[S2];
            if (c >= best[S]) continue;
            c += pair_time(nb, S1, S2, prec, cc);
            if (c < best[S]) {
                best[S] = c;
                split[S] = S1;
            }
        }
    }
    std::vector<std::array<uint64_t, 2>> pairs;  // post-order merges
    std::function<void(uint64_t)> rec = [&](uint64_t S) {
        if (popc(S) < 2) return;
        uint64_t S1 = split[S], S2 = S ^ S1;
        rec(S1);
        rec(S2);
        pairs.push_back({S1, S2});
    };
    rec(full);
    return pairs;
}

// Greedy: repeatedly merge the pair with the smallest predicted step time,
// preferring pairs that share a cut (an outer product only when nothing else
// is left).
std::vector<std::array<uint64_t, 2>> greedy_tree(const NetBits &nb, int prec, const CostConsts &cc) {
    std::vector<uint64_t> cur;
    for (int j = 0; j < nb.m; ++j) cur.push_back(1ull << j);
    std::vector<std::array<uint64_t, 2>> pairs;
    while (cur.size() > 1) {
        double bt = std::numeric_limits<double>::infinity();
        int bi = -1, bj = -1;
        bool bconn = false;
        for (size_t i = 0; i < cur.size(); ++i)
            for (size_t j = i + 1; j < cur.size(); ++j) {
                SubsetInfo x = subset_info(nb, cur[i]), y = subset_info(nb, cur[j]);
                bool conn = (x.cuts & y.cuts) != 0;
                double t = pair_time(nb, cur[i], cur[j], prec, cc);
                if ((conn && !bconn) || (conn == bconn && t < bt)) {
                    bt = t;
                    bi = (int)i;
                    bj = (int)j;
                    bconn = conn;
                }
            }
        pairs.push_back({cur[bi], cur[bj]});
        uint64_t merged = cur[bi] | cur[bj];
        cur.erase(cur.begin() + bj);
        cur[bi] = merged;
    }
    return pairs;
}

uint64_t mix64(uint64_t &x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// A random contraction tree: merge a uniformly drawn pair among those that
// share a cut (any pair once none do).
std::vector<std::array<uint64_t, 2>> random_tree(const NetBits &nb, uint64_t &rng) {
    std::vector<uint64_t> cur;
    for (int j = 0; j < nb.m; ++j) cur.push_back(1ull << j);
    std::vector<std::array<uint64_t, 2>> pairs;
    while (cur.size() > 1) {
        std::vector<std::pair<int, int>> conn, all;
        for (size_t i = 0; i < cur.size(); ++i)
            for (size_t j = i + 1; j < cur.size(); ++j) {
                all.push_back({(int)i, (int)j});
                if (subset_info(nb, cur[i]).cuts & subset_info(nb, cur[j]).cuts) conn.push_back({(int)i, (int)j});
            }
        const auto &pool = conn.empty() ? all : conn;
        auto pr = pool[mix64(rng) % pool.size()];
        pairs.push_back({cur[pr.first], cur[pr.second]});
        uint64_t merged = cur[pr.first] | cur[pr.second];
        cur.erase(cur.begin() + pr.second);
        cur[pr.first] = merged;
    }
    return pairs;
}

// Candidate trees for the learned planner: the optimum of the time, the
// multiply-add and the byte models (dynamic programming, m <= 14), greedy on
// the time model, then random trees; duplicates removed.
std::vector<std::vector<std::array<uint64_t, 2>>> candidate_trees(const NetBits &nb, int prec, const CostConsts &cc,
                                                                  int max_n, uint64_t seed) {
    std::vector<std::vector<std::array<uint64_t, 2>>> out;
    std::vector<std::vector<uint64_t>> seen;
    auto add = [&](std::vector<std::array<uint64_t, 2>> t) {
        std::vector<uint64_t> key;
        for (auto &p : t) key.push_back(p[0] | p[1]);
        std::sort(key.begin(), key.end());
        if (std::find(seen.begin(), seen.end(), key) != seen.end()) return;
        seen.push_back(key);
        out.push_back(std::move(t));
    };
    if (nb.m <= 14)
        for (int mode : {0, 1, 2}) {
            g_cost_mode = mode;
            add(exhaustive_tree(nb, prec, cc));
        }
    g_cost_mode = 0;
    add(greedy_tree(nb, prec, cc));
    uint64_t rng = seed;
    for (int tries = 0; (int)out.size() < max_n && tries < 20 * max_n; ++tries) add(random_tree(nb, rng));
    if ((int)out.size() > max_n) out.resize(max_n);
    return out;
}

std::vector<int32_t> pairs_to_order(const std::vector<std::array<uint64_t, 2>> &pairs, int m) {
    std::vector<uint64_t> sets;
    for (int j = 0; j < m; ++j) sets.push_back(1ull << j);
    std::vector<int32_t> ord;
    for (auto &pr : pairs) {
        ord.push_back((int32_t)(std::find(sets.begin(), sets.end(), pr[0]) - sets.begin()));
        ord.push_back((int32_t)(std::find(sets.begin(), sets.end(), pr[1]) - sets.begin()));
        sets.push_back(pr[0] | pr[1]);
    }
    return ord;
}

// SSA order (leaves 0..m-1, step s creates m+s) -> subset pairs
tqc_status order_to_pairs(const std::vector<std::array<int, 2>> &order, int m,
                          std::vector<std::array<uint64_t, 2>> *pairs) {
    if ((int)order.size() != m - 1) return fail(TQC_ERR_INVALID, "order must have m-1 steps");
    std::vector<uint64_t> sets(2 * m - 1, 0);
    std::vector<char> used(2 * m - 1, 0);
    for (int j = 0; j < m; ++j) sets[j] = 1ull << j;
    for (int s = 0; s < m - 1; ++s) {
        int a = order[s][0], b = order[s][1];
        if (a < 0 || b < 0 || a >= m + s || b >= m + s || a == b || used[a] || used[b])
            return fail(TQC_ERR_INVALID, "order step " + std::to_string(s) + " uses an invalid or consumed id");
        used[a] = used[b] = 1;
        sets[m + s] = sets[a] | sets[b];
        pairs->push_back({sets[a], sets[b]});
    }
    return TQC_OK;
}

struct Built {
    std::vector<TensorPlan> t;
    std::vector<StepPlan> s;
};

// Tensors and steps of a tree for a given free-qubit set and sliced cuts.
// `zplan`: scalar network for the total mass (no outputs, FP64, CUDA cores).
Built build_steps(const Plan &p, const NetBits &nb, const std::vector<std::array<uint64_t, 2>> &pairs,
                  int prec, bool zplan) {
    Built B;
    const Net &net = *p.net;
    std::vector<char> isfree(net.n_qubits, 0);
    if (!zplan)
        for (int q : p.free_qubits) isfree[q] = 1;
    auto make_tensor = [&](uint64_t leaves) {
        TensorPlan t;
        t.leaves = leaves;
        uint64_t cm = 0;
        for (int j = 0; j < p.m; ++j)
            if (leaves >> j & 1) {
                for (int q : net.nodes[j].out_qubits)
                    if (isfree[q]) t.qubits.push_back(q);
                for (int c : net.nodes[j].cut_ids) cm ^= 1ull << c;
            }
        std::sort(t.qubits.begin(), t.qubits.end());
        uint64_t open = cm & ~nb.sliced;
        for (int c = 0; c < 64; ++c)
            if (open >> c & 1) t.cuts.push_back(c);
        t.slice_dep = false;
        for (int c = 0; c < 64; ++c)
            if ((nb.sliced >> c & 1))
                for (int j = 0; j < p.m; ++j)
                    if ((leaves >> j & 1) && (nb.cutmask[j] >> c & 1)) t.slice_dep = true;
        return t;
    };
    for (int j = 0; j < p.m; ++j) B.t.push_back(make_tensor(1ull << j));
    std::vector<uint64_t> sets;
    for (int j = 0; j < p.m; ++j) sets.push_back(1ull << j);
    for (size_t s = 0; s < pairs.size(); ++s) {
        uint64_t x = pairs[s][0], y = pairs[s][1];
        int ia = (int)(std::find(sets.begin(), sets.end(), x) - sets.begin());
        int ib = (int)(std::find(sets.begin(), sets.end(), y) - sets.begin());
        TensorPlan c = make_tensor(x | y);
        sets.push_back(x | y);
        B.t.push_back(c);
        StepPlan st;
        const TensorPlan &ta = B.t[ia], &tb = B.t[ib];
        uint64_t ca = 0, cb = 0;
        for (int q : ta.cuts) ca |= 1ull << q;
        for (int q : tb.cuts) cb |= 1ull << q;
        uint64_t shared = ca & cb;
        int mb = (int)ta.qubits.size() + 2 * popc(ca & ~shared);
        int nbb = (int)tb.qubits.size() + 2 * popc(cb & ~shared);
        st.a = ia;
        st.b = ib;
        st.mb = mb;
        st.nb = nbb;
        if (mb < nbb) {  // rows = the larger operand
            std::swap(st.a, st.b);
            std::swap(st.mb, st.nb);
        }
        st.kb = 2 * popc(shared);
        st.c = (int)B.t.size() - 1;
        st.prec = zplan ? TQC_PREC_FP32 : step_prec(prec, st.mb, st.nb, st.kb);
        st.klass = zplan ? KC_SIMT : choose_class(st.mb, st.nb, st.kb, prec);
        st.final = (s + 1 == pairs.size());
        B.s.push_back(st);
    }
    // storage of every tensor: set by its consumer
    for (auto &t : B.t) t.storage = zplan ? ST_F64 : ST_F32;
    if (!zplan)
        for (auto &st : B.s) {
            int sto = ST_F32;
            if (st.klass == KC_UMMA) {
                if (st.prec == TQC_PREC_BF16) sto = ST_BF16;
                else if (st.prec == TQC_PREC_BF16X3) sto = ST_BF16X2;
                else sto = ST_TF32;
            }
            B.t[st.a].storage = sto;
            B.t[st.b].storage = sto;
        }
    return B;
}

// Layouts, top-down from the root (free qubits ascending = bin order).
void assign_layouts(Built &B, int m) {
    if (B.s.empty()) {
        // single node: its operand layout is the bin order
        TensorPlan &t = B.t[0];
        t.layout.modes.clear();
        for (int q : t.qubits) t.layout.modes.push_back({0, (int16_t)q});
        return;
    }
    TensorPlan &root = B.t.back();
    root.layout.modes.clear();
    for (int q : root.qubits) root.layout.modes.push_back({0, (int16_t)q});
    (void)m;
    std::vector<int> producer(B.t.size(), -1);  // step that writes each tensor
    for (size_t s = 0; s < B.s.size(); ++s) producer[(size_t)B.s[s].c] = (int)s;
    for (int s = (int)B.s.size() - 1; s >= 0; --s) {
        StepPlan &st = B.s[s];
        const Layout &LC = B.t[st.c].layout;
        TensorPlan &A = B.t[st.a];
        TensorPlan &Bt = B.t[st.b];
        std::vector<int> shared;
        std::set_intersection(A.cuts.begin(), A.cuts.end(), Bt.cuts.begin(), Bt.cuts.end(),
                              std::back_inserter(shared));
        // The shared cuts form the K field, the lowest bits of both operands;
        // their order is free as long as both operands agree.  Order it for
        // the step that writes the row operand (else the column operand): one
        // of its column-operand cuts first, then its row-operand cuts, so that
        // its epilogue's warp stores cover whole sectors -- four consecutive
        // columns per lane, consecutive rows in consecutive lanes.
        {
            const int t_in = producer[(size_t)st.a] >= 0 ? st.a : (producer[(size_t)st.b] >= 0 ? st.b : -1);
            if (t_in >= 0) {
                const StepPlan &ps = B.s[(size_t)producer[(size_t)t_in]];
                const std::vector<int> &rc = B.t[ps.a].cuts, &cc = B.t[ps.b].cuts;
                std::vector<int> cols, rows, rest;
                for (int c : shared) {
                    if (std::binary_search(cc.begin(), cc.end(), c)) cols.push_back(c);
                    else if (std::binary_search(rc.begin(), rc.end(), c)) rows.push_back(c);
                    else rest.push_back(c);
                }
                std::vector<int> ord;
                if (!cols.empty()) ord.push_back(cols[0]);
                ord.insert(ord.end(), rows.begin(), rows.end());
                if (cols.size() > 1) ord.insert(ord.end(), cols.begin() + 1, cols.end());
                ord.insert(ord.end(), rest.begin(), rest.end());
                shared = ord;
            }
        }
        std::vector<int> shared_sorted = shared;  // membership tests
        std::sort(shared_sorted.begin(), shared_sorted.end());
        // Tensor-core operands whose rows exceed 64 KB are K-blocked: the
        // lowest three shared cuts (64 elements) stay lowest, the row bits
        // follow, then the rest of K.  A 128-row copy box is then one
        // contiguous region instead of 128 rows strided across many pages.
        const int elem = st.prec == TQC_PREC_TF32 ? 4 : 2;
        st.kblk = st.klass == KC_UMMA && st.kb >= 6 && ((int64_t)elem << st.kb) > ((int64_t)1 << 16);
        const size_t n_low = st.kblk ? 3 : shared.size();
        auto make = [&](TensorPlan &T, uint64_t *mask) {
            std::vector<std::pair<int, Mode>> outer;  // (position in LC, mode)
            for (int q : T.qubits) {
                Mode md{0, (int16_t)q};
                outer.push_back({LC.pos(md), md});
            }
            for (int c : T.cuts)
                if (!std::binary_search(shared_sorted.begin(), shared_sorted.end(), c)) {
                    Mode md{1, (int16_t)c};
                    outer.push_back({LC.pos(md), md});
                }
            std::sort(outer.begin(), outer.end(), [](auto &x, auto &y) { return x.first < y.first; });
            T.layout.modes.clear();
            for (size_t i = 0; i < n_low; ++i) T.layout.modes.push_back({1, (int16_t)shared[i]});
            uint64_t mk = 0;
            for (auto &pm : outer) {
                T.layout.modes.push_back(pm.second);
                for (int b = 0; b < pm.second.bits(); ++b) mk |= 1ull << (pm.first + b);
            }
            for (size_t i = n_low; i < shared.size(); ++i) T.layout.modes.push_back({1, (int16_t)shared[i]});
            *mask = mk;
        };
        make(A, &st.maskR);
        make(Bt, &st.maskC);
    }
}

int64_t align256(int64_t x) { return (x + 255) & ~int64_t(255); }

// Workspace layout: every leaf operand and every intermediate result gets
// its own region (the final result goes to the caller's buffer, or to the
// FP64 slice accumulator).
int64_t assign_offsets(Built &B, bool zplan, int64_t *acc_off, bool need_acc, int64_t out_elems) {
    int64_t off = 0;
    size_t n = B.t.size();
    for (size_t i = 0; i < n; ++i) {
        TensorPlan &t = B.t[i];
        bool is_root = (i + 1 == n);
        int64_t elems = (int64_t)1 << t.nbits();
        int eb = storage_bytes(t.storage);
        if (t.storage == ST_BF16X2) eb = 2;
        t.plane_bytes = elems * eb;
        if (is_root && !zplan && !B.s.empty()) {
            t.offset = -1;  // caller's output / accumulator
            continue;
        }
        if (is_root && zplan) {
            t.offset = -1;  // Z slice slot
            continue;
        }
        if (B.s.empty() && !zplan) {  // single node: ingest straight to the output
            t.offset = -1;
            continue;
        }
        t.offset = off;
        off = align256(off + t.plane_bytes * (t.storage == ST_BF16X2 ? 2 : 1));
    }
    if (need_acc) {
        *acc_off = off;
        off = align256(off + 8 * out_elems);
    }
    return off;
}

std::string mode_str(const Layout &L) {
    std::ostringstream os;
    os << "[";
    for (size_t i = 0; i < L.modes.size(); ++i) {
        if (i) os << ",";
        os << "\"" << (L.modes[i].is_cut ? "c" : "q") << L.modes[i].id << "\"";
    }
    os << "]";
    return os.str();
}

const char *prec_name(int p) {
    switch (p) {
        case TQC_PREC_FP32: return "fp32";
        case TQC_PREC_TF32: return "tf32";
        case TQC_PREC_BF16: return "bf16";
        case TQC_PREC_BF16X3: return "bf16x3";
        default: return "auto";
    }
}

}  // namespace

// Plan features for the learned cost model: sums and maxima over steps of
// log2 M, N, K, log2 flops, log2 bytes; counts; slices; class mix.
std::vector<double> plan_features(const Plan &p) {
    std::vector<double> f(32, 0.0);
    double ns = (double)p.n_slices();
    CostConsts cc;
    double tot_flops = 0, tot_bytes = 0, max_fl = 0, max_by = 0, n_umma = 0, n_simt = 0;
    double smb = 0, snb = 0, skb = 0, mxm = 0, mxn = 0, mxk = 0, pred = 0, small_k = 0;
    for (auto &st : p.steps) {
        StepCost c = step_cost(st.mb, st.nb, st.kb, st.klass, st.prec, cc);
        tot_flops += 2 * c.macs;
        tot_bytes += c.bytes;
        max_fl = std::max(max_fl, 2 * c.macs);
        max_by = std::max(max_by, c.bytes);
        smb += st.mb;
        snb += st.nb;
        skb += st.kb;
        mxm = std::max(mxm, (double)st.mb);
        mxn = std::max(mxn, (double)st.nb);
        mxk = std::max(mxk, (double)st.kb);
        pred += c.time_s;
        (st.klass == KC_UMMA ? n_umma : n_simt) += 1;
        if (st.kb <= 4) small_k += 1;
    }
    auto lg = [](double x) { return std::log2(std::max(x, 1.0)); };
    int k = 0;
    f[k++] = lg(tot_flops * ns);
    f[k++] = lg(tot_bytes * ns);
    f[k++] = lg(max_fl);
    f[k++] = lg(max_by);
    f[k++] = smb / 8.0;
    f[k++] = snb / 8.0;
    f[k++] = skb / 8.0;
    f[k++] = mxm;
    f[k++] = mxn;
    f[k++] = mxk;
    f[k++] = (double)p.steps.size();
    f[k++] = lg(ns);
    f[k++] = n_umma;
    f[k++] = n_simt;
    f[k++] = small_k;
    f[k++] = (double)p.free_qubits.size();
    f[k++] = lg(pred * 1e9);
    // operand types: the share of the tensor-core steps in each (the plain
    // FP32 form has none)
    double n_prec[4] = {0, 0, 0, 0};  // BF16, BF16X3, TF32, FP32
    for (auto &st : p.steps) {
        if (st.klass != KC_UMMA) continue;
        n_prec[st.prec == TQC_PREC_BF16 ? 0 : st.prec == TQC_PREC_BF16X3 ? 1 : 2] += 1;
    }
    n_prec[3] = p.precision == TQC_PREC_FP32 ? 1.0 : 0.0;
    for (int i = 0; i < 3; ++i) f[k++] = n_umma > 0 ? n_prec[i] / n_umma : 0.0;
    f[k++] = n_prec[3];
    f[k++] = (double)p.m;
    f[k++] = (double)p.net->n_cuts;
    f[k++] = lg(p.ws_bytes);
    // final step shape
    if (!p.steps.empty()) {
        const StepPlan &fs = p.steps.back();
        f[k++] = fs.mb;
        f[k++] = fs.nb;
        f[k++] = fs.kb;
    }
    return f;
}

namespace {

constexpr int kAutoExhaustiveMax = 12;  // TQC_PLANNER_AUTO: exhaustive DP up to this many subcircuits

// Learned planner: plan every candidate tree completely (slicing, kernel
// classes, layouts), predict each plan's log time with the cost model on the
// GPU, keep the fastest.
constexpr double kLearnedWindow = 10.0;  // analytic-estimate window of the ranked candidates

tqc_status learned_tree(Net *net, const tqc_plan_opts &o, const NetBits &nb, int prec, const CostConsts &cc,
                        std::vector<std::array<uint64_t, 2>> *pairs, std::string *why) {
    if (!o.costmodel_path) {
        *why = "no cost-model path";
        return TQC_ERR_INVALID;
    }
    tqc_costmodel *cm = nullptr;
    if (costmodel_for_path(o.costmodel_path, &cm) != TQC_OK) {
        *why = tqc_last_error();
        return TQC_ERR_INVALID;
    }
    if (costmodel_n_in(cm) != (int)kPlanFeatures) {
        *why = "cost model expects another feature count";
        return TQC_ERR_INVALID;
    }
    auto cands = candidate_trees(nb, prec, cc, 24, 0x5EEDull + (uint64_t)nb.m);
    // Build every candidate (slicing to the budget); the analytic model is the
    // guard: only candidates within kLearnedWindow of its best estimate are
    // ranked, so the network is never asked about shapes far outside the
    // plans it was trained on.
    std::vector<Plan> built(cands.size());
    std::vector<char> valid(cands.size(), 0);
    double best_pred = std::numeric_limits<double>::infinity();
    for (size_t i = 0; i < cands.size(); ++i) {
        std::vector<int32_t> ord = pairs_to_order(cands[i], nb.m);
        tqc_plan_opts oc = o;
        oc.order = ord.data();
        oc.n_order = nb.m - 1;
        oc.planner = TQC_PLANNER_GREEDY;
        if (build_plan(net, oc, &built[i]) != TQC_OK) continue;
        valid[i] = 1;
        best_pred = std::min(best_pred, built[i].predicted_s);
    }
    std::vector<float> feats;
    std::vector<int> ok;
    for (size_t i = 0; i < cands.size(); ++i) {
        if (!valid[i] || built[i].predicted_s > kLearnedWindow * best_pred) continue;
        for (double f : plan_features(built[i])) feats.push_back((float)f);
        ok.push_back((int)i);
    }
    if (ok.empty()) {
        *why = "no valid candidate";
        return TQC_ERR_INVALID;
    }
    std::vector<float> pred(ok.size());
    if (costmodel_predict_host(cm, feats.data(), (int)ok.size(), pred.data()) != TQC_OK) {
        *why = tqc_last_error();
        return TQC_ERR_CUDA;
    }
    // the network predicts log(measured / analytic): add the analytic log time back
    for (size_t k = 0; k < ok.size(); ++k) pred[k] += (float)std::log(built[(size_t)ok[k]].predicted_s);
    size_t best = std::min_element(pred.begin(), pred.end()) - pred.begin();
    *pairs = cands[ok[best]];
    return TQC_OK;
}

}  // namespace

std::vector<std::vector<int32_t>> plan_candidate_orders(Net *net, const tqc_plan_opts &o, int max_n) {
    Plan tmp;
    tmp.net = net;
    tmp.m = (int)net->nodes.size();
    std::vector<char> isfree(net->n_qubits, 0);
    for (int q = 0; q < net->n_qubits; ++q)
        isfree[q] = !o.use_free_mask || (q < 64 ? (o.free_mask_lo >> q & 1) : (o.free_mask_hi >> (q - 64) & 1));
    for (int q = 0; q < net->n_qubits; ++q)
        if (isfree[q]) tmp.free_qubits.push_back(q);
    for (int i = 0; i < o.n_sliced; ++i) tmp.sliced.push_back(o.sliced_cuts[i]);
    NetBits nb = net_bits(tmp);
    CostConsts cc;
    std::vector<std::vector<int32_t>> out;
    if (tmp.m < 2) return out;
    for (auto &c : candidate_trees(nb, effective_prec(o.precision), cc, max_n, 0x5EEDull + (uint64_t)nb.m))
        out.push_back(pairs_to_order(c, tmp.m));
    return out;
}

tqc_status build_plan(Net *net, const tqc_plan_opts &o, Plan *p) {
    p->net = net;
    p->m = (int)net->nodes.size();
    if (net->n_cuts > 63) return fail(TQC_ERR_UNSUPPORTED, "more than 63 cuts");
    if (p->m > 63) return fail(TQC_ERR_UNSUPPORTED, "more than 63 subcircuits");
    // bin
    p->free_qubits.clear();
    for (int q = 0; q < net->n_qubits; ++q) {
        bool fr = !o.use_free_mask || (q < 64 ? (o.free_mask_lo >> q & 1) : (o.free_mask_hi >> (q - 64) & 1));
        if (fr) p->free_qubits.push_back(q);
    }
    if (net->n_qubits < 128 && net->n_qubits >= 64 && (o.free_mask_hi >> (net->n_qubits - 64)) != 0)
        return fail(TQC_ERR_INVALID, "free mask names qubits beyond n_qubits");
    if (net->n_qubits < 64 && (o.free_mask_lo >> net->n_qubits) != 0)
        return fail(TQC_ERR_INVALID, "free mask names qubits beyond n_qubits");
    if (p->free_qubits.size() > 40) return fail(TQC_ERR_UNSUPPORTED, "more than 40 free qubits in a bin");
    p->fixed_bits.assign(net->n_qubits, 0);
    if (o.fixed_bits)
        for (int q = 0; q < net->n_qubits; ++q) {
            if (o.fixed_bits[q] > 1) return fail(TQC_ERR_INVALID, "fixed_bits entries must be 0 or 1");
            p->fixed_bits[q] = o.fixed_bits[q];
        }
    p->precision = o.precision;
    if (p->precision < TQC_PREC_FP32 || p->precision > TQC_PREC_AUTO)
        return fail(TQC_ERR_INVALID, "unknown precision");
    int prec = effective_prec(p->precision);
    p->precision = prec;
    p->planner = o.planner;
    p->flags = o.flags;
    p->autotune = o.autotune;
    p->budget = o.mem_budget_bytes;
    p->sliced.clear();
    for (int i = 0; i < o.n_sliced; ++i) {
        int c = o.sliced_cuts[i];
        if (c < 0 || c >= net->n_cuts) return fail(TQC_ERR_INVALID, "sliced cut " + std::to_string(c) + " out of range");
        if (std::find(p->sliced.begin(), p->sliced.end(), c) == p->sliced.end()) p->sliced.push_back(c);
    }
    std::sort(p->sliced.begin(), p->sliced.end());

    CostConsts cc;
    NetBits nb = net_bits(*p);
    std::vector<std::array<uint64_t, 2>> pairs;
    p->order.clear();
    if (p->m > 1) {
        if (o.n_order > 0) {
            std::vector<std::array<int, 2>> ord;
            for (int i = 0; i < o.n_order; ++i) ord.push_back({o.order[2 * i], o.order[2 * i + 1]});
            tqc_status st = order_to_pairs(ord, p->m, &pairs);
            if (st != TQC_OK) return st;
            p->planner_used = "given";
        } else {
            int pl = o.planner;
            std::string prefix;
            if (pl == TQC_PLANNER_LEARNED) {
                // rank candidate plans with the learned cost model; the
                // exhaustive / greedy planner is the fallback
                std::string why;
                if (learned_tree(net, o, nb, prec, cc, &pairs, &why) == TQC_OK) p->planner_used = "learned";
                else prefix = "fallback (" + why + "): ";
            }
            if (pairs.empty()) {
                // exhaustive up to 12 subcircuits (planning under about 50 ms
                // there; measured 3% faster plans than greedy on 9-12)
                if (pl == TQC_PLANNER_AUTO || pl == TQC_PLANNER_LEARNED)
                    pl = p->m <= kAutoExhaustiveMax ? TQC_PLANNER_EXHAUSTIVE : TQC_PLANNER_GREEDY;
                if (pl == TQC_PLANNER_EXHAUSTIVE && p->m > 14)
                    return fail(TQC_ERR_UNSUPPORTED, "exhaustive planner limited to 14 subcircuits");
                pairs = pl == TQC_PLANNER_EXHAUSTIVE ? exhaustive_tree(nb, prec, cc) : greedy_tree(nb, prec, cc);
                p->planner_used = prefix + (pl == TQC_PLANNER_EXHAUSTIVE ? "exhaustive" : "greedy");
            }
        }
    } else {
        p->planner_used = "single";
    }

    // two-tier slicing: inputs first, then inputs + intermediates + FP64 sum
    auto mem_of = [&](const NetBits &b, bool inputs_only) {
        Plan tmp = *p;
        Built B = build_steps(tmp, b, pairs, prec, false);
        double in = 0, mid = 0;
        for (size_t i = 0; i < B.t.size(); ++i) {
            double sz = std::ldexp((double)storage_bytes(B.t[i].storage), B.t[i].nbits());
            if ((int)i < p->m) in += sz;
            else if (i + 1 < B.t.size()) mid += sz;
        }
        double acc = b.sliced ? 8.0 * (double)p->out_elems() : 0.0;
        return inputs_only ? in : in + mid + acc;
    };
    if (p->budget > 0 && p->m > 1) {
        for (int tier = 0; tier < 2; ++tier) {
            while (mem_of(nb, tier == 0) > (double)p->budget) {
                double best = std::numeric_limits<double>::infinity();
                int bc = -1;
                for (int c = 0; c < net->n_cuts; ++c) {
                    if (nb.sliced >> c & 1) continue;
                    NetBits t = nb;
                    t.sliced |= 1ull << c;
                    double mm = mem_of(t, tier == 0);
                    if (mm < best) {  // strictly smaller: ties keep the lowest cut id
                        best = mm;
                        bc = c;
                    }
                }
                if (bc < 0) return fail(TQC_ERR_OOM, "memory budget too small even with every cut sliced");
                nb.sliced |= 1ull << bc;
                p->sliced.push_back(bc);
            }
        }
        std::sort(p->sliced.begin(), p->sliced.end());
    }

    Built B = build_steps(*p, nb, pairs, prec, false);
    assign_layouts(B, p->m);
    bool need_acc = !p->sliced.empty() && p->m > 1;
    p->acc_offset = -1;
    p->ws_bytes = assign_offsets(B, false, &p->acc_offset, need_acc, p->out_elems());
    p->tensors = std::move(B.t);
    p->steps = std::move(B.s);
    // consecutive tensor-core steps whose layouts let the intermediate stay on chip
    if (!(p->flags & TQC_FLAG_NO_FUSE))
        for (size_t s = 0; s + 1 < p->steps.size(); ++s)
            if (!p->steps[s].fuse && fused_pair_ok(*p, s)) {
                p->steps[s].fuse = 1;
                p->steps[s + 1].fuse = 2;
            }

    NetBits zb = nb;  // Z uses the same slices; each slice adds its scalar
    Built Z = build_steps(*p, zb, pairs, prec, true);
    assign_layouts(Z, p->m);
    int64_t dummy = -1;
    p->zws_bytes = assign_offsets(Z, true, &dummy, false, 1);
    p->ztensors = std::move(Z.t);
    p->zsteps = std::move(Z.s);

    // SSA order of the chosen tree
    {
        std::vector<uint64_t> sets;
        for (int j = 0; j < p->m; ++j) sets.push_back(1ull << j);
        for (auto &pr : pairs) {
            int a = (int)(std::find(sets.begin(), sets.end(), pr[0]) - sets.begin());
            int b = (int)(std::find(sets.begin(), sets.end(), pr[1]) - sets.begin());
            p->order.push_back({a, b});
            sets.push_back(pr[0] | pr[1]);
        }
    }

    // totals
    double ns = (double)p->n_slices();
    p->flops = 0;
    p->bytes = 0;
    p->predicted_s = 0;
    for (auto &st : p->steps) {
        StepCost c = step_cost(st.mb, st.nb, st.kb, st.klass, st.prec, cc);
        p->flops += 2.0 * c.macs * ns;
        p->bytes += c.bytes * ns;
        p->predicted_s += c.time_s * ns;
    }
    // leaf ingest: read the bin-restricted rows once, write the operand
    for (int j = 0; j < p->m; ++j) {
        double e = std::ldexp(1.0, p->tensors[j].nbits());
        p->bytes += e * (8.0 + storage_bytes(p->tensors[j].storage)) * (p->tensors[j].slice_dep ? ns : 1.0);
    }

    p->describe_json = plan_describe(*p);
    return TQC_OK;
}

// Plan summary as JSON (current state: tiles reflect the autotuner once run).
std::string plan_describe(const Plan &pl) {
    const Plan *p = &pl;
    const Net *net = p->net;
    std::ostringstream os;
    os << "{\"m\":" << p->m << ",\"n_qubits\":" << net->n_qubits << ",\"n_cuts\":" << net->n_cuts
       << ",\"free\":" << p->free_qubits.size() << ",\"precision\":\"" << prec_name(p->precision)
       << "\",\"planner\":\"" << p->planner_used << "\",\"tuned\":" << p->tuned
       << ",\"ready\":" << (p->ready ? 1 : 0) << ",\"sliced\":[";
    for (size_t i = 0; i < p->sliced.size(); ++i) os << (i ? "," : "") << p->sliced[i];
    os << "],\"order\":[";
    for (size_t i = 0; i < p->order.size(); ++i)
        os << (i ? "," : "") << "[" << p->order[i][0] << "," << p->order[i][1] << "]";
    os << "],\"steps\":[";
    for (size_t i = 0; i < p->steps.size(); ++i) {
        auto &st = p->steps[i];
        os << (i ? "," : "") << "{\"a\":" << st.a << ",\"b\":" << st.b << ",\"c\":" << st.c << ",\"log2_m\":" << st.mb
           << ",\"log2_n\":" << st.nb << ",\"log2_k\":" << st.kb << ",\"class\":\""
           << (st.klass == KC_UMMA ? "tcgen05" : "simt") << "\",\"prec\":\""
           << (st.klass == KC_UMMA ? prec_name(st.prec) : "fp32") << "\",\"out_layout\":" << mode_str(p->tensors[st.c].layout)
           << ",\"mask_r\":" << st.maskR << ",\"mask_c\":" << st.maskC << ",\"tile\":" << st.tile
           << ",\"ksplit\":" << st.ksplit << ",\"kblk\":" << (st.kblk ? 1 : 0) << ",\"fuse\":" << st.fuse << "}";
    }
    os << "],\"layouts\":[";
    for (size_t i = 0; i < p->tensors.size(); ++i) os << (i ? "," : "") << mode_str(p->tensors[i].layout);
    // kernel launches of one contract once the total mass is cached, and of
    // the total-mass network when the tensors changed
    const int64_t z_launches = ((int64_t)p->m + (int64_t)p->zsteps.size()) * p->n_slices() + 1;
    int64_t launches = 0;
    if (p->m == 1) launches += 1;
    else {
        for (int j = 0; j < p->m; ++j) launches += p->tensors[j].slice_dep ? p->n_slices() : 1;
        for (auto &st : p->steps)  // a K-split step adds its reduce pass; a fused pair is one launch
            if (st.fuse != 2) launches += (p->tensors[st.c].slice_dep ? p->n_slices() : 1) * (st.ksplit > 1 ? 2 : 1);
        if (p->n_slices() > 1) launches += 1;
    }
    os << "],\"launches_per_contract\":" << launches << ",\"total_mass_launches\":" << z_launches;
    // how tqc_contract_states runs this plan (plans with no free qubits only)
    const char *sf = "none";
    if (p->free_qubits.empty()) sf = states_fused_floats(*p) >= 0 ? "fused" : "per-state";
    os << ",\"states_form\":\"" << sf << "\"";
    os << ",\"reused_leaves\":" << p->reused_leaves << ",\"reused_steps\":" << p->reused_steps;
    char buf[256];
    std::snprintf(buf, sizeof buf, ",\"flops\":%.6g,\"bytes\":%.6g,\"predicted_s\":%.6g,\"ws_bytes\":%lld}", p->flops,
                  p->bytes, p->predicted_s, (long long)p->ws_bytes);
    os << buf;
    return os.str();
}

}  // namespace tqc
