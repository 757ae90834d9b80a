"""Batched persistent launch: many plans of uneven sizes in one kernel, under
a captured CUDA graph, with bounded device waits."""
import numpy as np
import pytest

import oracle
from gen import Network, Node, tensors, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2502_03445_gb300 import tqc  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def uneven_networks():
    nets = [tensors.shape_matched_network(12 + k, 2 + k % 4, 3 + k, 12 if k == 4 else 9, seed=3000 + k)
            for k in range(6)]
    outs = [[0, 3, 6, 9, 12, 15], [1, 4, 7, 10, 13], [2, 5, 8, 11, 14]]
    nets.append(tensors.pseudo_physical_network(16, [(0, 1)] * 3 + [(1, 2)] * 3, outs, 3100))  # tensor-core steps
    rng = np.random.Generator(np.random.PCG64(5))
    nets.append(Network(5, 0, [Node([4, 0, 2, 1, 3], [], [], rng.random(32))]))                # one subcircuit
    return nets


def term_scale(net):
    """Mean absolute term mass per state: the reconstruction with |T_j| in
    place of T_j, summed over all states, over 2^n."""
    a = Network(net.n_qubits, net.n_cuts,
                [Node(nd.out_qubits, nd.cut_ids, nd.cut_role, np.abs(nd.data)) for nd in net.nodes])
    return float(oracle.total_mass(a)) / float(1 << net.n_qubits)


def prepared(nets, precs):
    hs, plans, outs, want = [], [], [], []
    for net, prec in zip(nets, precs):
        h = tqc.Network(net)
        p = tqc.Plan(h, precision=prec)
        o = torch.empty(p.out_elems, dtype=torch.float32, device="cuda")
        z = p.contract(o, want_z=True)        # allocates the workspace and caches Z
        hs.append(h)
        plans.append(p)
        outs.append(torch.full_like(o, float("nan")))
        zo = oracle.total_mass(net)
        want.append((oracle.recon_bin(net) / zo, term_scale(net) / abs(zo)))
    return hs, plans, outs, want


FP32_ATOL = 1e-5
TC_TV = 1e-3


def check(outs, want, plans):
    """Each plan at its own form's gate: plans whose steps run in FP32 or
    split BF16 (FP32-class products) meet 1e-5 absolute per probability and,
    as a second check, stay within 1e-4 of the largest probability or within
    n_steps * 2^-12 of the mean absolute term mass per state, whichever is
    larger (signed terms cancel: a K = 4^8 step sums 65536 of them); a plan
    with a TF32 step meets the 1e-3 total-variation gate of the tensor-core
    forms."""
    for o, (w, scale), p in zip(outs, want, plans):
        got = o.cpu().numpy().astype(np.float64)
        err = np.abs(got - w)
        steps = p.describe()["steps"]
        precs = {st["prec"] for st in steps if st["class"] == "tcgen05"}
        assert "bf16" not in precs
        if "tf32" in precs:
            tv = 0.5 * err.sum() / np.abs(w).sum()
            assert tv <= TC_TV, (tv, precs)
        else:
            assert err.max() <= FP32_ATOL, err.max()
            bound = max(1e-4 * np.abs(w).max(), max(len(steps), 1) * 2.0 ** -12 * scale)
            assert err.max() <= bound, (err.max(), bound, precs)


@pytest.mark.parametrize("mode", ["fp32", "auto", "mixed"])
def test_batch_matches_oracle(mode):
    nets = uneven_networks()
    precs = {"fp32": ["fp32"] * len(nets), "auto": ["auto"] * len(nets),
             "mixed": ["fp32", "bf16x3", "tf32", "auto", "fp32", "bf16x3", "tf32", "fp32"]}[mode]
    hs, plans, outs, want = prepared(nets, precs)
    tqc.contract_batch(plans, outs)
    tqc.batch_status()
    check(outs, want, plans)
    for p in plans:
        p.close()


@pytest.mark.parametrize("tail_s", [0.0, 1e-6, 3e-6])
def test_batch_large_steps_after_the_persistent_kernel(tail_s):
    """Steps predicted to take at least tail_s run as ordinary step launches
    after the persistent kernel (0: every step; the kernel only ingests),
    also when the whole batch is replayed from a CUDA graph."""
    nets = uneven_networks()
    hs, plans, outs, want = prepared(nets, ["auto"] * len(nets))
    tqc.batch_tail_threshold(tail_s)
    try:
        tqc.contract_batch(plans, outs)
        tqc.batch_status()
        check(outs, want, plans)
        launches, tail_steps = tqc.batch_launches()
        if tail_s == 0.0:
            assert tail_steps == sum(len(p.describe()["steps"]) for p in plans)
        assert launches >= 1 + (tail_steps > 0) and launches <= 1 + 2 * tail_steps
        for o in outs:
            o.fill_(float("nan"))
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            tqc.contract_batch(plans, outs, stream=s)
        g.replay()
        torch.cuda.synchronize()
        tqc.batch_status()
        check(outs, want, plans)
    finally:
        tqc.batch_tail_threshold(16e-6)
    for p in plans:
        p.close()


def test_batch_large_step_timeout_is_reported_once():
    """With every step after the persistent kernel (threshold 0) and the
    tensor-core step stall hook on, the large steps' bounded waits give up:
    tqc_batch_status reports it and clears every plan's error word, and a
    clean rerun reports nothing and matches the oracle."""
    nets = uneven_networks()
    hs, plans, outs, want = prepared(nets, ["auto"] * len(nets))
    assert any(st["class"] == "tcgen05" for p in plans for st in p.describe()["steps"])
    tqc.batch_tail_threshold(0.0)
    try:
        tqc.step_inject_stall(True)
        try:
            tqc.contract_batch(plans, outs)
            with pytest.raises(tqc.TqcError) as ei:
                tqc.batch_status()
        finally:
            tqc.step_inject_stall(False)
        assert ei.value.status == tqc.ERR_TIMEOUT
        tqc.contract_batch(plans, outs)
        tqc.batch_status()
        check(outs, want, plans)
    finally:
        tqc.batch_tail_threshold(16e-6)
    for p in plans:
        p.close()


def test_batch_tail_threshold_rejects_negative():
    with pytest.raises(tqc.TqcError):
        tqc.batch_tail_threshold(-1.0)


def test_batch_autotuned_tiles():
    """Plans tuned by the autotuner: the batch runs each tensor-core step at
    the tile width the autotuner chose, with the same results."""
    nets = uneven_networks()
    hs, plans, outs, want = [], [], [], []
    for net in nets:
        h = tqc.Network(net)
        p = tqc.Plan(h, precision="auto", autotune=1)
        o = torch.empty(p.out_elems, dtype=torch.float32, device="cuda")
        p.contract(o)
        assert p.describe()["tuned"] == 1
        hs.append(h)
        plans.append(p)
        outs.append(torch.full_like(o, float("nan")))
        zo = oracle.total_mass(net)
        want.append((oracle.recon_bin(net) / zo, term_scale(net) / abs(zo)))
    tqc.contract_batch(plans, outs)
    tqc.batch_status()
    check(outs, want, plans)
    for p in plans:
        p.close()


def test_batch_k_blocked_operands():
    """Plans whose deep steps read K-blocked operands (rows over 64 KB)."""
    nets = [tensors.pseudo_physical_network(14, [(0, 1)] * 8, [list(range(7)), list(range(7, 14))], 3200),
            tensors.pseudo_physical_network(15, [(0, 1)] * 8, [list(range(8)), list(range(8, 15))], 3201)]
    precs = ["bf16x3", "tf32"]
    hs, plans, outs_, want = prepared(nets, precs)
    for p in plans:
        assert any(st["kblk"] for st in p.describe()["steps"])
    tqc.contract_batch(plans, outs_)
    tqc.batch_status()
    check(outs_, want, plans)
    for p in plans:
        p.close()


def test_batch_under_cuda_graph():
    nets = uneven_networks()
    hs, plans, outs, want = prepared(nets, ["auto"] * len(nets))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        tqc.contract_batch(plans, outs, stream=s)   # first call builds the work list
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        tqc.contract_batch(plans, outs, stream=s)
    for o in outs:
        o.fill_(float("nan"))
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    tqc.batch_status()
    check(outs, want, plans)


def test_batch_bounded_wait_reports_timeout():
    """A wait that nothing can satisfy gives up after about a second; the
    error is reported and the context stays usable."""
    nets = uneven_networks()[:3]
    hs, plans, outs, want = prepared(nets, ["fp32"] * 3)
    tqc.batch_inject_stall(True)
    try:
        tqc.contract_batch(plans, outs)
        with pytest.raises(tqc.TqcError) as ei:
            tqc.batch_status()
        assert ei.value.status == tqc.ERR_TIMEOUT
    finally:
        tqc.batch_inject_stall(False)
    tqc.contract_batch(plans, outs)
    tqc.batch_status()
    check(outs, want, plans)


def test_batch_rejects_sliced_plans():
    net = tensors.shape_matched_network(12, 3, 5, 9, seed=3200)
    h = tqc.Network(net)
    p = tqc.Plan(h, precision="fp32", sliced=[1])
    o = torch.empty(p.out_elems, dtype=torch.float32, device="cuda")
    p.contract(o)
    with pytest.raises(tqc.TqcError) as ei:
        tqc.contract_batch([p], [o])
    assert ei.value.status == tqc.ERR_UNSUPPORTED


def test_batch_full_recipe_sampled():
    """The batched workload at full size: 256 networks (n 16-28, 2-8
    subcircuits, 2-12 cuts, 1.0e10 outputs), one persistent launch replayed
    from a CUDA graph; four sampled states per network against oracle A.
    Raw probabilities (no renormalisation: the Gaussian tensors' total mass
    can be near zero), errors measured against each network's mean absolute
    term mass per state (the reconstruction with |T_j|), bound
    n_steps * 2^-12 of it (split BF16 or FP32 products, FP32 accumulation)."""
    nets, _ = workloads.batch_recipe(256)
    hs, plans, outs = [], [], []
    for net in nets:
        h = tqc.Network(net, dtype=tqc.F32)
        p = tqc.Plan(h, precision="auto", flags=tqc.FLAG_NO_RENORM)
        o = torch.empty(p.out_elems, dtype=torch.float32, device="cuda")
        p.contract(o)
        hs.append(h)
        plans.append(p)
        outs.append(torch.full_like(o, float("nan")))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        tqc.contract_batch(plans, outs, stream=s)
    s.synchronize()
    for o in outs:
        o.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        tqc.contract_batch(plans, outs, stream=s)
    g.replay()
    torch.cuda.synchronize()
    tqc.batch_status()
    rng = np.random.Generator(np.random.PCG64(77))
    worst = 0.0
    for net, p, o in zip(nets, plans, outs):
        idx = sorted(set(int(i) for i in rng.integers(0, 1 << net.n_qubits, size=4)))
        want = oracle.recon_states(net, idx)
        got = o[torch.tensor(idx, device="cuda")].double().cpu().numpy()
        a = Network(net.n_qubits, net.n_cuts,
                    [Node(nd.out_qubits, nd.cut_ids, nd.cut_role, np.abs(nd.data)) for nd in net.nodes])
        scale = oracle.total_mass(a) / float(1 << net.n_qubits)
        n_steps = max(len(p.describe()["steps"]), 1)
        rel = float(np.abs(got - want).max()) / (n_steps * 2.0 ** -12 * scale)
        worst = max(worst, rel)
        assert rel <= 1.0, (net.n_qubits, net.n_cuts, rel)
    print(f"batch256: worst error / bound {worst:.3e}")
    for p in plans:
        p.close()
    for h in hs:
        h.close()
