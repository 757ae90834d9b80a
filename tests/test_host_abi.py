"""Host-side checks of the C ABI (no GPU): exports, validation, planner
arithmetic (the worked example's 144 vs 768 multiplications, §III-C),
slicing under a memory budget (§III-E-2)."""
import json
import re

import numpy as np
import pytest

from gen import Network, Node, tensors, workloads
from conftest import golden_path, ROOT
from paper_2502_03445_gb300 import tqc


def header_functions():
    with open(f"{ROOT}/include/tqc.h") as f:
        src = f.read()
    return sorted(set(re.findall(r"TQC_API\s+[\w\s\*]+?\b(tqc_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = tqc.lib()
    declared = header_functions()
    assert declared and set(declared) == set(tqc.EXPORTS)
    for name in declared:
        assert hasattr(L, name), name


def shape_net(n_qubits, edges, outs):
    """Shape-only network with cut i = edges[i] = (upstream, downstream)."""
    m = len(outs)
    cuts = [[] for _ in range(m)]
    for cid, (a, b) in enumerate(edges):
        cuts[a].append((cid, 0))
        cuts[b].append((cid, 1))
    nodes = []
    for j in range(m):
        cl = sorted(cuts[j])
        nodes.append(Node(list(outs[j]), [c for c, _ in cl], [r for _, r in cl],
                          np.zeros((4 ** len(cl)) << len(outs[j]))))
    return Network(n_qubits, len(edges), nodes)


def test_worked_example_144_vs_768():
    with open(golden_path("worked_example_cost.json")) as f:
        g = json.load(f)
    net = shape_net(4, [tuple(e) for e in g["edges"]], [[0], [1], [2], [3]])
    h = tqc.Network(net, shape_only=True)
    # one reconstructed state: every qubit fixed (an empty free set)
    p = tqc.Plan(h, precision="fp32", free_qubits=[], order=g["order"])
    info = p.info()
    assert info["flops"] / 2 == g["tn_multiplications_per_state"] == 144
    steps = [2 ** (p.step(i)["log2_m"] + p.step(i)["log2_n"] + p.step(i)["log2_k"]) for i in range(3)]
    assert steps == g["step_multiplications_per_state"]
    # brute force: 4^|E| terms, m-1 multiplications each
    assert 4 ** 4 * 3 == g["bruteforce_multiplications_per_state"]
    # the exhaustive planner never does worse than the worked order
    pe = tqc.Plan(h, precision="fp32", free_qubits=[], planner=tqc.PLANNER_EXHAUSTIVE)
    assert pe.info()["flops"] <= info["flops"]
    p.close(), pe.close(), h.close()


@pytest.mark.parametrize("n_cuts", [1, 3, 5])
def test_two_subcircuits_cost_equals_bruteforce(n_cuts):
    """With two subcircuits the one step sums all 4^|E| terms (§III-D)."""
    net = shape_net(2, [(0, 1)] * n_cuts, [[0], [1]])
    h = tqc.Network(net, shape_only=True)
    p = tqc.Plan(h, precision="fp32", free_qubits=[])
    assert p.info()["flops"] / 2 == 4 ** n_cuts * (2 - 1)


def test_step_shapes_are_consistent():
    net = workloads.grid30()
    h = tqc.Network(net, shape_only=True)
    for prec in ("fp32", "bf16", "bf16x3", "tf32"):
        p = tqc.Plan(h, precision=prec)
        d = p.describe()
        assert d["m"] == 4 and d["n_cuts"] == 10 and len(d["steps"]) == 3
        last = d["steps"][-1]
        assert last["log2_m"] + last["log2_n"] == 30 and last["log2_k"] % 2 == 0
        for st in d["steps"]:
            assert st["log2_m"] >= st["log2_n"]
        p.close()
    h.close()


def test_exhaustive_never_worse_than_greedy():
    for seed in range(6):
        net = tensors.shape_matched_network(20, 5 + seed % 3, 8 + seed, 10, seed=300 + seed)
        h = tqc.Network(net, shape_only=True)
        pe = tqc.Plan(h, precision="bf16", planner=tqc.PLANNER_EXHAUSTIVE)
        pg = tqc.Plan(h, precision="bf16", planner=tqc.PLANNER_GREEDY)
        assert pe.describe()["predicted_s"] <= pg.describe()["predicted_s"] * (1 + 1e-12)
        pe.close(), pg.close(), h.close()


def test_auto_plans_exhaustively_up_to_12_subcircuits():
    """TQC_PLANNER_AUTO takes the exhaustive DP for m <= 12 (its plan is the
    DP's, never predicted slower than greedy's) and greedy above."""
    for seed in range(9500, 9506):
        net = workloads.planner_network(seed, "m9")
        assert 9 <= len(net.nodes) <= 12
        h = tqc.Network(net, shape_only=True)
        pa = tqc.Plan(h, planner=tqc.PLANNER_AUTO)
        pe = tqc.Plan(h, planner=tqc.PLANNER_EXHAUSTIVE)
        pg = tqc.Plan(h, planner=tqc.PLANNER_GREEDY)
        da, de, dg = pa.describe(), pe.describe(), pg.describe()
        assert da["planner"] == "exhaustive"
        assert da["predicted_s"] == de["predicted_s"] <= dg["predicted_s"] * (1 + 1e-12)
        pa.close(), pe.close(), pg.close(), h.close()
    net = tensors.random_shape_network(26, 13, 15, 10, seed=77, max_node_cuts=6)
    h = tqc.Network(net, shape_only=True)
    p = tqc.Plan(h, planner=tqc.PLANNER_AUTO)
    assert p.describe()["planner"] == "greedy"
    p.close(), h.close()


def test_small_k_workload_cases_have_their_named_shapes():
    """The small-K bench cases (gen.workloads.SMALLK_CASES) plan to a single
    CUDA-core step of the named M, N, K, with the named bits lowest."""
    for case in workloads.SMALLK_CASES:
        m, rest = case.split("x")
        n, k = rest.split("k")[0], rest.split("k")[1].split("_")[0]
        net = workloads.smallk_network(case)
        h = tqc.Network(net, shape_only=True)
        p = tqc.Plan(h, precision="fp32")
        (st,) = p.describe()["steps"]
        assert (st["log2_m"], st["log2_n"], 1 << st["log2_k"]) == (int(m), int(n), int(k)), (case, st)
        assert st["class"] == "simt"
        if case.endswith("rows_low"):
            assert st["mask_r"] & 0xF == 0xF
        elif case.endswith("cols_low"):
            assert st["mask_c"] & 0xF == 0xF
        else:
            assert st["mask_r"] & 0xF not in (0, 0xF)
        p.close(), h.close()


def test_slicing_under_budget():
    net = workloads.grid30()
    h = tqc.Network(net, shape_only=True)
    free = list(range(16))
    p0 = tqc.Plan(h, precision="fp32", free_qubits=free)
    assert p0.info()["n_slices"] == 1
    ws0 = p0.describe()["ws_bytes"]
    p1 = tqc.Plan(h, precision="fp32", free_qubits=free, mem_budget=ws0 // 4)
    d1 = p1.describe()
    assert p1.info()["n_slices"] >= 4 and d1["sliced"]
    assert d1["ws_bytes"] <= ws0 // 4 + 4096        # budget met up to alignment padding
    assert p1.info()["flops"] >= p0.info()["flops"]  # slicing never saves arithmetic
    with pytest.raises(tqc.TqcError) as ei:
        tqc.Plan(h, precision="fp32", free_qubits=free, mem_budget=64)
    assert ei.value.status == tqc.ERR_OOM
    # forced slicing is honoured
    p2 = tqc.Plan(h, precision="fp32", free_qubits=free, sliced=[3, 7])
    assert p2.describe()["sliced"] == [3, 7] and p2.info()["n_slices"] == 16


def _expect_invalid(net, fragment):
    with pytest.raises(tqc.TqcError) as ei:
        tqc.Network(net, shape_only=True)
    assert ei.value.status == tqc.ERR_INVALID
    assert fragment in str(ei.value), str(ei.value)


def test_validation_errors_name_the_culprit():
    good = shape_net(3, [(0, 1), (1, 2)], [[0], [1], [2]])
    tqc.Network(good, shape_only=True).close()
    bad = shape_net(3, [(0, 1), (1, 2)], [[0], [1], [1]])
    _expect_invalid(bad, "subcircuit 2: output qubit 1 already output by subcircuit 1")
    bad = shape_net(3, [(0, 1), (1, 2)], [[0], [1], []])
    _expect_invalid(bad, "qubit 2 is not an output")
    bad = shape_net(3, [(0, 1), (1, 2)], [[0], [1], [2]])
    bad.nodes[2].cut_role = [0]      # cut 1 now has two upstream ends
    _expect_invalid(bad, "cut 1: two upstream ends")
    bad = shape_net(3, [(0, 1), (1, 2)], [[0], [1], [2]])
    bad.nodes[0].cut_ids = [0, 0]
    bad.nodes[0].cut_role = [0, 1]
    bad.nodes[1].cut_ids = [1]
    bad.nodes[1].cut_role = [0]
    _expect_invalid(bad, "joins a subcircuit to itself")


def test_bad_order_is_rejected():
    net = shape_net(3, [(0, 1), (1, 2)], [[0], [1], [2]])
    h = tqc.Network(net, shape_only=True)
    with pytest.raises(tqc.TqcError) as ei:
        tqc.Plan(h, order=[[0, 1], [0, 2]])
    assert ei.value.status == tqc.ERR_INVALID


def test_contract_on_shape_only_network_fails_cleanly():
    net = shape_net(2, [(0, 1)], [[0], [1]])
    h = tqc.Network(net, shape_only=True)
    p = tqc.Plan(h)
    st = tqc.lib().tqc_contract(p.handle, None, 16, tqc.F32, None, None)
    assert st == tqc.ERR_INVALID


@pytest.mark.parametrize("prec,cuts,expect", [("bf16x3", 8, 1), ("bf16", 8, 1), ("tf32", 8, 1),
                                              ("bf16x3", 7, 0), ("tf32", 7, 0), ("fp32", 8, 0)])
def test_k_blocked_layout_rule(prec, cuts, expect):
    """Tensor-core operands with rows over 64 KB are K-blocked: the three
    lowest shared cuts (64 elements), then the row bits, then the other
    shared cuts.  Rows of up to 64 KB, and CUDA-core operands, stay K-major
    (every shared cut below the row bits).  Both operands list the shared
    cuts in the same order."""
    net = Network(16, cuts, [Node(list(range(8)), list(range(cuts)), [0] * cuts, None),
                             Node(list(range(8, 16)), list(range(cuts)), [1] * cuts, None)])
    h = tqc.Network(net, shape_only=True)
    p = tqc.Plan(h, precision=prec)
    d = p.describe()
    st = d["steps"][-1]
    assert st["log2_k"] == 2 * cuts and st["kblk"] == expect, st
    for t in (st["a"], st["b"]):
        kinds = [m[0] for m in d["layouts"][t]]
        if expect:
            assert kinds == ["c"] * 3 + ["q"] * 8 + ["c"] * (cuts - 3), d["layouts"][t]
        else:
            assert kinds == ["c"] * cuts + ["q"] * 8, d["layouts"][t]
    cuts_a = [m for m in d["layouts"][st["a"]] if m[0] == "c"]
    cuts_b = [m for m in d["layouts"][st["b"]] if m[0] == "c"]
    assert cuts_a == cuts_b
    p.close()
    h.close()


def test_auto_precision_is_chosen_per_step():
    """TQC_PREC_AUTO: TF32 for a step that split BF16 would leave bound by
    the tensor pipe, split BF16 for HBM-bound tensor-core steps (grid30's
    final step writes 4.3 GB for 5.5e11 flops), FP32 on CUDA cores."""
    # deep K: M = 2^11, N = 2^10, K = 4^7 -- 69 GFLOP per 210 MB
    deep = tqc.Network(shape_net(21, [(0, 1)] * 7, [list(range(11)), list(range(11, 21))]), shape_only=True)
    p = tqc.Plan(deep)
    d = p.describe()
    assert d["precision"] == "auto"
    assert [(s["class"], s["prec"], s["log2_k"]) for s in d["steps"]] == [("tcgen05", "tf32", 14)]
    assert p.step(0)["precision"] == tqc.PREC_TF32
    p.close(), deep.close()
    g30 = tqc.Network(workloads.grid30(), shape_only=True)
    p = tqc.Plan(g30)
    d = p.describe()
    last = d["steps"][-1]
    assert last["class"] == "tcgen05" and last["prec"] == "bf16x3", d["steps"]
    assert last["log2_m"] + last["log2_n"] == 30
    for s in d["steps"]:
        if s["class"] == "tcgen05":
            m, n, k = 2 ** s["log2_m"], 2 ** s["log2_n"], 2 ** s["log2_k"]
            bound = 2 * m * n * k * 3 / 1.6e15 > 4 * (m * k + n * k + m * n) / 6.79e12
            assert s["prec"] == ("tf32" if bound else "bf16x3"), s
    # a forced precision applies to every tensor-core step
    for prec in ("bf16x3", "tf32"):
        pf = tqc.Plan(g30, precision=prec)
        assert {s["prec"] for s in pf.describe()["steps"] if s["class"] == "tcgen05"} == {prec}
        pf.close()
    p.close(), g30.close()


def test_auto_precision_on_the_tensor_bound_bins():
    """The 48-qubit QAOA and 64-qubit grid bins (32 GB budget): AUTO runs
    their tensor-bound steps in TF32, the rest in split BF16."""
    for net in (workloads.qaoa48(0), workloads.grid64_bin(0, 0)):
        h = tqc.Network(net, shape_only=True)
        p = tqc.Plan(h, mem_budget=32 << 30)
        steps = p.describe()["steps"]
        tc = [s for s in steps if s["class"] == "tcgen05"]
        assert steps[-1]["prec"] == "tf32", steps
        assert {s["prec"] for s in tc} == {"tf32", "bf16x3"}, steps
        for s in tc:
            m, n, k = 2 ** s["log2_m"], 2 ** s["log2_n"], 2 ** s["log2_k"]
            bound = 2 * m * n * k * 3 / 1.6e15 > 4 * (m * k + n * k + m * n) / 6.79e12
            assert s["prec"] == ("tf32" if bound else "bf16x3"), s
        p.close(), h.close()
