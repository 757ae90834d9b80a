// Cut finder (§VI) and the cost report of a plan (§III-C, §VIII).
//
// Finding wire cuts is a constrained partition of the circuit's two-qubit
// gates (§VI-A).  Greedy Graph Growing (Alg. 2) starts from one partition per
// two-qubit gate and repeatedly merges the two partitions joined by the edge
// of least merging cost (Alg. 3), summed from three metrics by the rule of
// Table I: the trial partition's width w and size s against the QPU limits
// (hard: x / T, not allowed above T) and the largest number of contraction
// edges K between it and a neighbour against a threshold K_t (soft: x / T,
// 4^{x - T} + 1 above T).  It stops when no edge is valid (cost at most
// Q_max).  One-qubit gates then join an adjacent two-qubit gate.
//
// The objective of §V-VI, T = T_QPU + T_classical (Eq. cut_objective), picks
// among the partitions found for a range of thresholds K_t: T_QPU follows
// Eq. qpu_runtime; T_classical is the planner's own estimate of contracting
// the resulting network (its step-time model, or the learned cost model in
// place of the FLOP count over FLOP/s of Eq. classical_runtime).
//
// Readings (the paper leaves these open): a partition's width is its number
// of wire segments (a wire that leaves and re-enters comes back on a new
// qubit); its size is its number of two-qubit gates; K of two neighbouring
// partitions is the number of distinct cuts touching either (inner plus
// outer contraction edges, §III-C); every merging cost is recomputed after
// each merge; ties go to the lowest edge (pairs of gate indices in order);
// the merged partition keeps the lower label; one-qubit gates join the next
// two-qubit gate on their wire, else the previous one, else subcircuit 0;
// subcircuits are numbered by their first gate; shots = 2^w limited to
// [2^shots_log2_min, 2^shots_log2_max] (§V); a subcircuit's depth is the
// number of layers of its gates scheduled as early as possible.
#include <algorithm>
#include <cmath>
#include <limits>
#include <string>
#include <vector>

#include "tqc_internal.h"

namespace tqc {

namespace {

constexpr double kInf = std::numeric_limits<double>::infinity();

struct Circuit {
    int n = 0;
    std::vector<std::array<int, 2>> gates;  // (q0, q1), q1 = -1 for a one-qubit gate
    std::vector<int> multi;                 // two-qubit gate ids
    std::vector<int> dense;                 // gate id -> index into multi (-1 for one-qubit gates)
    std::vector<std::vector<int>> wires;    // per qubit: its two-qubit gates (dense indices) in order
    std::vector<std::array<int, 2>> edges;  // (earlier, later) dense indices, sorted, unique
};

Circuit make_circuit(int n, int n_gates, const int32_t *gq) {
    Circuit c;
    c.n = n;
    c.dense.assign((size_t)n_gates, -1);
    c.wires.assign((size_t)n, {});
    for (int g = 0; g < n_gates; ++g) {
        c.gates.push_back({gq[2 * g], gq[2 * g + 1]});
        if (gq[2 * g + 1] >= 0) {
            c.dense[(size_t)g] = (int)c.multi.size();
            c.multi.push_back(g);
            c.wires[(size_t)gq[2 * g]].push_back(c.dense[(size_t)g]);
            c.wires[(size_t)gq[2 * g + 1]].push_back(c.dense[(size_t)g]);
        }
    }
    for (auto &seq : c.wires)
        for (size_t i = 1; i < seq.size(); ++i)
            if (seq[i - 1] != seq[i]) c.edges.push_back({seq[i - 1], seq[i]});
    std::sort(c.edges.begin(), c.edges.end());
    c.edges.erase(std::unique(c.edges.begin(), c.edges.end()), c.edges.end());
    return c;
}

double table_cost(int x, int t, bool hard) {
    if (x <= t) return (double)x / (double)t;
    return hard ? kInf : std::ldexp(1.0, 2 * (x - t)) + 1.0;
}

// Merging cost Q_e of joining labels la < lb (Alg. 3); scratch arrays sized
// to the gate count.
double merging_cost(const Circuit &c, const std::vector<int> &lab, const std::vector<int> &size, int la, int lb,
                    int w_max, int s_max, int k_t, std::vector<int> &ncut, std::vector<int> &between) {
    std::fill(ncut.begin(), ncut.end(), 0);
    std::fill(between.begin(), between.end(), 0);
    int width = 0;
    for (const auto &seq : c.wires) {
        int prev = -1;
        for (int g : seq) {
            int L = lab[(size_t)g];
            if (L == lb) L = la;
            if (L == prev) continue;
            if (L == la) ++width;
            if (prev >= 0) {  // a cut between prev and L
                ++ncut[(size_t)prev];
                ++ncut[(size_t)L];
                if (prev == la) ++between[(size_t)L];
                if (L == la) ++between[(size_t)prev];
            }
            prev = L;
        }
    }
    int k_trial = 0;
    for (size_t N = 0; N < between.size(); ++N)
        if (between[N] > 0 && (int)N != la) k_trial = std::max(k_trial, ncut[(size_t)la] + ncut[N] - between[N]);
    return table_cost(width, w_max, true) + table_cost(size[(size_t)la] + size[(size_t)lb], s_max, true) +
           table_cost(k_trial, k_t, false);
}

// Alg. 2: a label per two-qubit gate (dense index -> label).
std::vector<int> greedy_graph_growing(const Circuit &c, int w_max, int s_max, int k_t, double q_max) {
    const size_t G = c.multi.size();
    std::vector<int> lab(G), size(G, 1), ncut(G), between(G);
    for (size_t g = 0; g < G; ++g) lab[g] = (int)g;
    for (;;) {
        double best = kInf;
        int ba = -1, bb = -1;
        for (const auto &e : c.edges) {
            int la = lab[(size_t)e[0]], lb = lab[(size_t)e[1]];
            if (la == lb) continue;
            if (la > lb) std::swap(la, lb);
            const double q = merging_cost(c, lab, size, la, lb, w_max, s_max, k_t, ncut, between);
            if (q < kInf && q <= q_max && q < best) {
                best = q;
                ba = la;
                bb = lb;
            }
        }
        if (ba < 0) return lab;
        for (auto &l : lab)
            if (l == bb) l = ba;
        size[(size_t)ba] += size[(size_t)bb];
        size[(size_t)bb] = 0;
    }
}

// Subcircuit of every gate, numbered by first gate.
std::vector<int> full_partition(const Circuit &c, const std::vector<int> &lab) {
    const int n_gates = (int)c.gates.size();
    std::vector<int> part((size_t)n_gates, -1);
    for (size_t i = 0; i < c.multi.size(); ++i) part[(size_t)c.multi[i]] = lab[i];
    for (int q = 0; q < c.n; ++q) {
        std::vector<int> mg;  // two-qubit gate ids on the wire, in order
        for (int d : c.wires[(size_t)q]) mg.push_back(c.multi[(size_t)d]);
        for (int g = 0; g < n_gates; ++g) {
            const auto &gt = c.gates[(size_t)g];
            if (gt[1] >= 0 || gt[0] != q) continue;
            auto it = std::upper_bound(mg.begin(), mg.end(), g);
            if (it != mg.end()) part[(size_t)g] = lab[(size_t)c.dense[(size_t)*it]];
            else if (!mg.empty()) part[(size_t)g] = lab[(size_t)c.dense[(size_t)mg.back()]];
        }
    }
    std::vector<int> renum(c.multi.size() + 1, -1);
    int next = 0;
    for (int g = 0; g < n_gates; ++g) {
        const int l = part[(size_t)g];
        if (l >= 0 && renum[(size_t)l] < 0) renum[(size_t)l] = next++;
    }
    for (auto &l : part) l = l >= 0 ? renum[(size_t)l] : 0;
    return part;
}

struct SubInfo {
    int width = 0, up = 0, down = 0, depth = 0;
    std::vector<int> outs;          // output qubits
    std::vector<int> cuts;          // cut ids
    std::vector<int8_t> roles;      // 0 upstream, 1 downstream
};

// Subcircuits of a gate partition: a wire is cut wherever consecutive gates
// on it sit in different subcircuits (cuts numbered in time order); a wire
// without gates is a qubit of subcircuit 0.
std::vector<SubInfo> subcircuits(const Circuit &c, const std::vector<int> &part, int *n_cuts) {
    int m = 1;
    for (int p : part) m = std::max(m, p + 1);
    std::vector<SubInfo> s((size_t)m);
    std::vector<int> cur((size_t)c.n, -1);
    std::vector<std::vector<int>> layer((size_t)m, std::vector<int>((size_t)c.n, 0));
    int nc = 0;
    for (size_t g = 0; g < c.gates.size(); ++g) {
        const int sb = part[g];
        const int qs[2] = {c.gates[g][0], c.gates[g][1]};
        int lvl = 0;
        for (int q : qs) {
            if (q < 0) continue;
            if (cur[(size_t)q] < 0) {
                ++s[(size_t)sb].width;
            } else if (cur[(size_t)q] != sb) {
                ++s[(size_t)sb].width;
                SubInfo &u = s[(size_t)cur[(size_t)q]];
                ++u.up;
                u.cuts.push_back(nc);
                u.roles.push_back(0);
                ++s[(size_t)sb].down;
                s[(size_t)sb].cuts.push_back(nc);
                s[(size_t)sb].roles.push_back(1);
                ++nc;
                layer[(size_t)sb][(size_t)q] = 0;  // a new local qubit, initialised by the cut
            }
            cur[(size_t)q] = sb;
            lvl = std::max(lvl, layer[(size_t)sb][(size_t)q]);
        }
        ++lvl;
        for (int q : qs)
            if (q >= 0) layer[(size_t)sb][(size_t)q] = lvl;
        s[(size_t)sb].depth = std::max(s[(size_t)sb].depth, lvl);
    }
    for (int q = 0; q < c.n; ++q) {
        if (cur[(size_t)q] < 0) {
            ++s[0].width;
            s[0].outs.push_back(q);
        } else {
            s[(size_t)cur[(size_t)q]].outs.push_back(q);
        }
    }
    *n_cuts = nc;
    return s;
}

double qpu_runtime(const std::vector<SubInfo> &subs, const tqc_cut_opts &o) {
    double t = 0;
    for (const SubInfo &s : subs) {
        const int lg = std::min(std::max(s.width, o.shots_log2_min), o.shots_log2_max);
        t += std::pow(3.0, s.up) * std::pow(4.0, s.down) * std::ldexp(1.0, lg) * (s.depth * o.t_gate + o.t_meas);
    }
    return t / std::max(1, o.n_qpus);
}

// The network of a partition (shape only, no device memory).
Net shape_net(int n, const std::vector<SubInfo> &subs, int n_cuts) {
    Net net;
    net.n_qubits = n;
    net.n_cuts = n_cuts;
    net.cut_nodes.assign((size_t)n_cuts, {-1, -1});
    for (size_t j = 0; j < subs.size(); ++j) {
        Node nd;
        nd.out_qubits = subs[j].outs;
        nd.cut_ids = subs[j].cuts;
        nd.cut_role = subs[j].roles;
        nd.elems = (int64_t)1 << std::min<int64_t>(62, (int64_t)nd.out_qubits.size() + 2 * (int64_t)nd.cut_ids.size());
        for (size_t d = 0; d < nd.cut_ids.size(); ++d) net.cut_nodes[(size_t)nd.cut_ids[d]][nd.cut_role[d]] = (int)j;
        net.nodes.push_back(std::move(nd));
    }
    return net;
}

}  // namespace

// T_classical of a network: the planner's estimated contraction time for the
// bin of the lowest `free` qubits, corrected by the learned cost model when
// one is given; also the per-state multiplications of the brute force
// (4^|E| (m - 1)) and of the plan's order on a single state.
tqc_status classical_estimate(Net *net, const tqc_cut_opts &o, double *t_classical, double *cutqc, double *tqc_mults) {
    const int m = (int)net->nodes.size();
    *cutqc = std::ldexp((double)std::max(m - 1, 0), 2 * net->n_cuts);
    if (net->n_cuts > 63 || m > 63) {
        *t_classical = kInf;
        *tqc_mults = kInf;
        return TQC_OK;
    }
    tqc_plan_opts po;
    tqc_plan_opts_default(&po);
    po.precision = o.precision;
    po.use_free_mask = 1;
    const int f = std::min(std::min(o.cost_free_qubits, net->n_qubits), 40);
    for (int q = 0; q < f; ++q) {
        if (q < 64) po.free_mask_lo |= 1ull << q;
        else po.free_mask_hi |= 1ull << (q - 64);
    }
    Plan p;
    tqc_status st = build_plan(net, po, &p);
    if (st != TQC_OK) return st;
    double t = p.predicted_s;
    if (o.costmodel_path) {
        tqc_costmodel *cm = nullptr;
        st = costmodel_for_path(o.costmodel_path, &cm);
        if (st != TQC_OK) return st;
        std::vector<float> feats;
        for (double x : plan_features(p)) feats.push_back((float)x);
        float y = 0;
        st = costmodel_predict_host(cm, feats.data(), 1, &y);
        if (st != TQC_OK) return st;
        t *= std::exp((double)y);  // the model predicts log(measured / analytic)
    }
    *t_classical = t;
    // the same order on one state (no free qubits): the paper's per-state count
    tqc_plan_opts ps = po;
    ps.free_mask_lo = ps.free_mask_hi = 0;
    ps.precision = TQC_PREC_FP32;
    std::vector<int32_t> ord;
    for (auto &pr : p.order) {
        ord.push_back(pr[0]);
        ord.push_back(pr[1]);
    }
    ps.n_order = (int32_t)p.order.size();
    ps.order = ord.data();
    Plan one;
    st = build_plan(net, ps, &one);
    if (st != TQC_OK) return st;
    *tqc_mults = one.flops / 2.0;
    return TQC_OK;
}

tqc_status find_cuts(int n, int n_gates, const int32_t *gq, const tqc_cut_opts &o, int32_t *gate_part,
                     tqc_cut_result *res) {
    for (int g = 0; g < n_gates; ++g) {
        const int a = gq[2 * g], b = gq[2 * g + 1];
        if (a < 0 || a >= n || b >= n || b == a || b < -1)
            return fail(TQC_ERR_INVALID, "gate " + std::to_string(g) + ": bad qubits");
    }
    if (o.w_max < 2 || o.s_max < 1) return fail(TQC_ERR_INVALID, "w_max must be >= 2 and s_max >= 1");
    if (o.shots_log2_min < 0 || o.shots_log2_max < o.shots_log2_min || o.shots_log2_max > 60)
        return fail(TQC_ERR_INVALID, "bad shot limits");
    const Circuit c = make_circuit(n, n_gates, gq);
    const double q_max = o.q_max > 0 ? o.q_max : kInf;
    const int k_lo = o.k_t > 0 ? o.k_t : 1, k_hi = o.k_t > 0 ? o.k_t : std::max(1, o.k_sweep_max);
    double best_t = kInf;
    bool found = false;
    for (int kt = k_lo; kt <= k_hi; ++kt) {
        std::vector<int> lab = greedy_graph_growing(c, o.w_max, o.s_max, kt, q_max);
        std::vector<int> part = full_partition(c, lab);
        int nc = 0;
        std::vector<SubInfo> subs = subcircuits(c, part, &nc);
        int wmax = 0;  // above w_max only through wires without two-qubit gates (subcircuit 0)
        for (auto &s : subs) wmax = std::max(wmax, s.width);
        Net net = shape_net(n, subs, nc);
        double t_cl = kInf, cq = 0, tm = 0;
        tqc_status st = classical_estimate(&net, o, &t_cl, &cq, &tm);
        if (st != TQC_OK) return st;
        const double t_q = qpu_runtime(subs, o);
        const double t = t_q + t_cl;
        if (!found || t < best_t) {
            found = true;
            best_t = t;
            std::copy(part.begin(), part.end(), gate_part);
            res->n_sub = (int32_t)subs.size();
            res->n_cuts = nc;
            res->k_t = kt;
            res->max_width = wmax;
            res->t_qpu = t_q;
            res->t_classical = t_cl;
            res->t_total = t;
            res->cutqc_mults = cq;
            res->tensorqc_mults = tm;
        }
    }
    return found ? TQC_OK : fail(TQC_ERR_INVALID, "empty threshold range");
}

}  // namespace tqc

struct tqc_plan {
    tqc::Plan p;
};

using namespace tqc;

extern "C" {

void tqc_cut_opts_default(tqc_cut_opts *o) {
    if (!o) return;
    *o = tqc_cut_opts{};
    o->w_max = 16;
    o->s_max = 1 << 20;
    o->k_t = 0;
    o->k_sweep_max = 16;
    o->q_max = 0;
    o->t_gate = 1e-7;
    o->t_meas = 1e-6;
    o->shots_log2_min = 10;
    o->shots_log2_max = 20;
    o->n_qpus = 10;
    o->cost_free_qubits = 20;
    o->precision = TQC_PREC_AUTO;
    o->costmodel_path = nullptr;
}

tqc_status tqc_find_cuts(int32_t n_qubits, int32_t n_gates, const int32_t *gate_qubits, const tqc_cut_opts *opts,
                         int32_t *gate_part, tqc_cut_result *result) {
    if (n_qubits < 1 || n_qubits > 128 || n_gates < 0) return fail(TQC_ERR_INVALID, "bad circuit size");
    if ((n_gates > 0 && (!gate_qubits || !gate_part)) || !result) return fail(TQC_ERR_INVALID, "NULL argument");
    tqc_cut_opts o;
    tqc_cut_opts_default(&o);
    if (opts) o = *opts;
    *result = tqc_cut_result{};
    try {
        return find_cuts(n_qubits, n_gates, gate_qubits, o, gate_part, result);
    } catch (const std::exception &ex) {
        return fail(TQC_ERR_OOM, std::string("cut finder: ") + ex.what());
    }
}

tqc_status tqc_plan_cost_report(tqc_plan_t plan, tqc_cost_report *out) {
    if (!plan || !out) return fail(TQC_ERR_INVALID, "NULL argument");
    const Plan &p = plan->p;
    Net *net = p.net;
    const int m = p.m;
    *out = tqc_cost_report{};
    out->cutqc_mults_per_state = std::ldexp((double)std::max(m - 1, 0), 2 * net->n_cuts);
    out->plan_mults = p.flops / 2.0;
    out->plan_mults_per_state = p.flops / 2.0 / (double)p.out_elems();
    // the plan's order on one state (no free qubits, no slicing): the
    // per-state count of §III-C and the largest step's contraction edges
    tqc_plan_opts ps;
    tqc_plan_opts_default(&ps);
    ps.use_free_mask = 1;
    ps.precision = TQC_PREC_FP32;
    std::vector<int32_t> ord;
    for (auto &pr : p.order) {
        ord.push_back(pr[0]);
        ord.push_back(pr[1]);
    }
    ps.n_order = (int32_t)p.order.size();
    ps.order = ord.empty() ? nullptr : ord.data();
    Plan one;
    tqc_status st;
    try {
        st = build_plan(net, ps, &one);
    } catch (const std::exception &ex) {
        return fail(TQC_ERR_OOM, std::string("cost report: ") + ex.what());
    }
    if (st != TQC_OK) return st;
    out->tensorqc_mults_per_state = one.flops / 2.0;
    int kmax = 0;
    for (auto &stp : one.steps) kmax = std::max(kmax, (stp.mb + stp.nb + stp.kb) / 2);
    out->k_max = kmax;
    out->tn_upper_bound = std::ldexp((double)m, 2 * kmax);
    out->ratio = out->tensorqc_mults_per_state > 0 ? out->cutqc_mults_per_state / out->tensorqc_mults_per_state : 0.0;
    return TQC_OK;
}

}  // extern "C"
