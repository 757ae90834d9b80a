"""The library's cut finder (tqc_find_cuts) and cost report
(tqc_plan_cost_report), host only.

* the partition equals the oracle's (oracle/cutfind.py, Alg. 2/3, Table I)
  gate for gate on the hand-derived fixture and on seeded random circuits,
  and T_QPU equals the oracle's Eq. qpu_runtime;
* T_classical is the planner's estimate for the network the partition
  cuts out (rebuilt here with the input generator's wire cutter);
* a threshold sweep keeps the least T_QPU + T_classical (Eq. cut_objective);
* the cost report reproduces the worked example's 144 / 768 multiplications
  per state (§III-C) and Eq. tn_upper_bound."""
import json
import math

import numpy as np
import pytest

from conftest import golden_path
from gen import Network, Node, cutter, statevector as sv, circuits
from oracle import cutfind as cf
from paper_2502_03445_gb300 import tqc


def load():
    with open(golden_path("cutfind_line3.json")) as f:
        g = json.load(f)
    return g["n_qubits"], [tuple(x) for x in g["gates"]], g


def lib_qmax(v):
    return 0.0 if v == math.inf or v == "inf" else float(v)


@pytest.mark.parametrize("case", range(4))
def test_matches_the_hand_derived_run(case):
    n, gates, g = load()
    c = g["cases"][case]
    part, r = tqc.find_cuts(n, gates, w_max=c["w_max"], s_max=c["s_max"], k_t=c["k_t"], q_max=lib_qmax(c["q_max"]),
                            n_qpus=1)
    assert part == c["partition"]
    assert r["n_cuts"] == c["n_cuts"] and r["n_sub"] == max(part) + 1
    if "t_qpu" in c:
        assert abs(r["t_qpu"] - c["t_qpu"]) <= 1e-15


def random_circuit(seed, n, n2q):
    rng = np.random.Generator(np.random.PCG64(seed))
    gates = []
    for _ in range(n2q):
        if rng.random() < 0.3:
            gates.append((int(rng.integers(n)),))
        a = int(rng.integers(n - 1))
        b = a + 1 if rng.random() < 0.7 else int(rng.integers(a + 1, n))
        gates.append((a, b) if rng.random() < 0.5 else (b, a))
    return gates


CASES = [(1, 6, 14, 4, 6, 3, math.inf), (2, 8, 20, 5, 8, 4, 3.0), (3, 10, 30, 6, 12, 5, math.inf),
         (4, 7, 18, 4, 5, 2, 2.5), (5, 9, 24, 5, 40, 6, math.inf), (6, 12, 40, 6, 10, 4, math.inf),
         (7, 14, 50, 7, 30, 5, 2.9)]


@pytest.mark.parametrize("seed,n,n2q,w_max,s_max,k_t,q_max", CASES)
def test_matches_the_oracle(seed, n, n2q, w_max, s_max, k_t, q_max):
    gates = random_circuit(seed, n, n2q)
    part, r = tqc.find_cuts(n, gates, w_max=w_max, s_max=s_max, k_t=k_t, q_max=lib_qmax(q_max), n_qpus=3)
    want = cf.full_partition(n, gates, cf.greedy_graph_growing(n, gates, w_max, s_max, k_t, q_max))
    assert part == want
    subs, n_cuts = cf.subcircuits(n, gates, part)
    assert r["n_cuts"] == n_cuts and r["n_sub"] == len(subs)
    assert r["max_width"] == max(s[0] for s in subs)
    assert r["t_qpu"] == pytest.approx(cf.qpu_runtime(subs, n_qpus=3), rel=1e-13)
    assert r["cutqc_mults"] == 4.0 ** n_cuts * (len(subs) - 1)


def shape_network(n, gates, part):
    """The network a partition cuts out, from the input generator's cutter."""
    cc = cutter.cut_circuit(n, [("g", qs, None) for qs in gates], part)
    edges, outs = cutter.network_shape(cc)
    m = len(outs)
    cuts = [[] for _ in range(m)]
    for cid, (a, b) in enumerate(edges):
        cuts[a].append((cid, 0))
        cuts[b].append((cid, 1))
    nodes = [Node(list(outs[j]), [c for c, _ in sorted(cuts[j])], [r for _, r in sorted(cuts[j])],
                  np.zeros((4 ** len(cuts[j])) << len(outs[j]))) for j in range(m)]
    return Network(n, len(edges), nodes)


@pytest.mark.parametrize("seed", [2, 3, 6, 7])
def test_classical_estimate_is_the_planners(seed):
    _, n, n2q, w_max, s_max, k_t, q_max = CASES[seed - 1]
    gates = random_circuit(seed, n, n2q)
    part, r = tqc.find_cuts(n, gates, w_max=w_max, s_max=s_max, k_t=k_t, q_max=lib_qmax(q_max), cost_free_qubits=8)
    if r["n_cuts"] > 63:      # beyond what the library contracts: an infinite estimate
        assert r["t_classical"] == math.inf
        return
    net = shape_network(n, gates, part)
    h = tqc.Network(net, shape_only=True)
    p = tqc.Plan(h, free_qubits=list(range(8)))
    assert r["t_classical"] == pytest.approx(p.describe()["predicted_s"], rel=1e-5)   # JSON keeps 6 digits
    assert r["tensorqc_mults"] == pytest.approx(p.cost_report()["tensorqc_mults_per_state"], rel=1e-12)
    assert r["t_total"] == pytest.approx(r["t_qpu"] + r["t_classical"], rel=1e-12)
    p.close()
    h.close()


def test_threshold_sweep_keeps_the_least_total_runtime():
    n, gates = circuits.qaoa_regular(14, 77)
    gq = [tuple(qs) for _, qs, _ in gates]
    part, best = tqc.find_cuts(n, gq, w_max=8, k_t=0, k_sweep_max=8, cost_free_qubits=10)
    totals = [tqc.find_cuts(n, gq, w_max=8, k_t=k, cost_free_qubits=10)[1]["t_total"] for k in range(1, 9)]
    assert best["t_total"] == min(totals)
    assert best["k_t"] == 1 + int(np.argmin(totals))
    assert best["max_width"] <= 8


def worked_example_plan():
    with open(golden_path("worked_example_cost.json")) as f:
        g = json.load(f)
    edges = [tuple(e) for e in g["edges"]]
    cuts = [[] for _ in range(4)]
    for cid, (a, b) in enumerate(edges):
        cuts[a].append((cid, 0))
        cuts[b].append((cid, 1))
    nodes = [Node([j], [c for c, _ in cuts[j]], [r for _, r in cuts[j]], np.zeros((4 ** len(cuts[j])) << 1))
             for j in range(4)]
    h = tqc.Network(Network(4, len(edges), nodes), shape_only=True)
    return g, h, tqc.Plan(h, precision="fp32", order=g["order"])


def test_cost_report_worked_example():
    g, h, p = worked_example_plan()
    r = p.cost_report()
    assert r["cutqc_mults_per_state"] == g["bruteforce_multiplications_per_state"] == 768
    assert r["tensorqc_mults_per_state"] == g["tn_multiplications_per_state"] == 144
    assert r["ratio"] == pytest.approx(768 / 144)
    assert r["k_max"] == 3 and r["tn_upper_bound"] == 4 ** 3 * 4
    assert r["tensorqc_mults_per_state"] <= r["tn_upper_bound"]
    # the bin of every qubit: 16 states share the work
    assert r["plan_mults"] == pytest.approx(16 * r["plan_mults_per_state"])
    p.close()
    h.close()


def test_found_cuts_are_valid_wire_cuts():
    """The subcircuits of a found partition reconstruct the uncut circuit:
    exact tensors of the cut circuit (input generator) through the FP64
    oracle equal the statevector's probabilities."""
    import oracle
    from gen import tensors
    n, gates = circuits.qaoa_regular(10, 5)
    gq = [tuple(qs) for _, qs, _ in gates]
    part, r = tqc.find_cuts(n, gq, w_max=6, k_t=0, k_sweep_max=6, cost_free_qubits=10)
    assert r["n_sub"] >= 2 and r["n_cuts"] >= 1 and r["max_width"] <= 6
    net = tensors.exact_network(cutter.cut_circuit(n, gates, part))
    np.testing.assert_allclose(oracle.recon_bin(net), sv.probabilities(n, gates), atol=1e-12)
