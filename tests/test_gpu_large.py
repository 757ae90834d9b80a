"""Full-size workloads, checked through the C ABI against the FP64 oracle.

* 48-qubit QAOA p=1 (3-regular graph, 5 subcircuits of width <= 16, 16-24
  cuts), one bin of 2^24 states, contracted with the memory budget forcing
  slicing: the final step is a tensor-core GEMM with K = 4^9..4^11.
* The 64-qubit grid shape (6 subcircuits, width <= 20, 27 cuts), a stream of
  bins of 2^24 states: one plan, new node tensors uploaded per bin.
* The bench workload itself: the 30-qubit grid shape, the full 2^30 bin, in
  the launch configuration bench.py times (checked with oracle A).

The oracle cannot produce 2^24 probabilities at these cut counts, so each
test checks (i) sampled states one by one with oracle B, and (ii) properties
that hold at any size: the bin's total mass Z (FP64 on the device) against
the oracle's, and the sum of all 2^24 outputs against Z.

Errors are measured against the scale of the terms, s = sum over the bin of
the reconstruction with |T_j| in place of T_j, divided by 2^F (the mean
absolute term mass per state): probabilities of pseudo-physical networks
are signed sums whose terms cancel, so |P| alone says nothing about the
rounding error.  Bound per state: n_steps * 2^-12 * s.  Each step rounds
its products to about 2^-16 relative (split BF16; 2^-24 for FP32) and
accumulates K terms in FP32, whose randomly signed rounding errors grow like
sqrt(K) * 2^-24 <= 2^-13 for K <= 2^22; the FP64 slice sum adds nothing
visible.  The absolute FP32 tolerance (1e-5 per probability) is asserted as
well."""
import functools

import numpy as np
import pytest

import oracle
from gen import Network, Node, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2502_03445_gb300 import tqc  # noqa: E402

FP32_ATOL = 1e-5
BUDGET = 32 << 30          # device bytes: forces slicing of both networks


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@functools.lru_cache(maxsize=None)
def qaoa48():
    return workloads.qaoa48(0)


@functools.lru_cache(maxsize=None)
def grid64(b):
    return workloads.grid64_bin(0, b)


def abs_scale(net):
    a = Network(net.n_qubits, net.n_cuts,
                [Node(nd.out_qubits, nd.cut_ids, nd.cut_role, np.abs(nd.data)) for nd in net.nodes])
    return float(oracle.total_mass(a)) / float(1 << net.n_qubits)


def sample(n_free, k, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return sorted(set(int(i) for i in rng.integers(0, 1 << n_free, size=k)))


def check_result(net, got, z, d, idx, label):
    """got: raw (unnormalised) FP64 copy of the device output."""
    z_or = oracle.total_mass(net)
    s = abs_scale(net)
    n_steps = len(d["steps"])
    # total mass: an FP64 scalar network on the device
    assert abs(z - z_or) <= 1e-9 * abs(z_or) + 1e-12 * s * (1 << net.n_qubits), (z, z_or)
    # the sum of every output equals Z (error: 2^F states x the per-state bound, but signed
    # rounding errors average out; the bound kept here is the per-state one x sqrt(2^F))
    tot = float(got.sum())
    tol_sum = n_steps * 2.0 ** -12 * s * np.sqrt(float(1 << net.n_qubits))
    want = oracle.recon_states_elim(net, idx)
    err = np.abs(got[idx] - want)
    print(f"{label}: slices={d.get('sliced')} steps={[(t['log2_m'], t['log2_n'], t['log2_k'], t['class']) for t in d['steps']]}"
          f" Z={z:.6e} (oracle {z_or:.6e}) sum-Z={tot - z_or:.3e} (tol {tol_sum:.3e})"
          f" max|err|={err.max():.3e} scale={s:.3e} err/scale={err.max() / s:.3e} max|P|={np.abs(want).max():.3e}")
    assert abs(tot - z_or) <= tol_sum, (tot, z_or, tol_sum)
    assert err.max() <= FP32_ATOL
    assert err.max() <= n_steps * 2.0 ** -12 * s, (err.max(), s)


def contract_raw(plan):
    out = torch.empty(plan.out_elems, dtype=torch.float32, device="cuda")
    z = plan.contract(out, want_z=True)
    torch.cuda.synchronize()
    return out.double().cpu().numpy(), z


@pytest.mark.parametrize("prec", ["auto", "fp32"])
def test_qaoa48_bin_full_size(prec):
    net = qaoa48()
    h = tqc.Network(net)
    p = tqc.Plan(h, precision=prec, mem_budget=BUDGET, flags=tqc.FLAG_NO_RENORM)
    d = p.describe()
    assert d["sliced"], "the budget must force slicing"
    if prec == "auto":
        assert d["steps"][-1]["class"] == "tcgen05" and d["steps"][-1]["log2_k"] >= 16
    got, z = contract_raw(p)
    check_result(net, got, z, d, sample(24, 24, 4), f"qaoa48/{prec}")
    p.close()
    h.close()


def test_grid64_bin_stream():
    """One plan, bins streamed by uploading each bin's node tensors."""
    first = grid64(0)
    h = tqc.Network(first)
    p = tqc.Plan(h, precision="auto", mem_budget=BUDGET, flags=tqc.FLAG_NO_RENORM)
    d = p.describe()
    assert d["sliced"]
    for b in range(3):
        net = grid64(b)
        if b:
            for j, nd in enumerate(net.nodes):
                assert nd.out_qubits == first.nodes[j].out_qubits and nd.cut_ids == first.nodes[j].cut_ids
                h.upload(j, nd.data)
        got, z = contract_raw(p)
        check_result(net, got, z, d, sample(24, 2 if b < 2 else 0, 50 + b) or [0], f"grid64/bin{b}")
    p.close()
    h.close()


@pytest.mark.parametrize("prec", ["auto", "fp32"])
def test_grid30_full_bin_sampled(prec):
    """bench.py's workload and launch configuration: every qubit free, the
    default plan (split-BF16 tensor-core steps with the direct and staged
    epilogues, or the plain FP32 form), renormalised FP32 output."""
    net = workloads.grid30(0)
    h = tqc.Network(net)
    p = tqc.Plan(h, precision=prec)
    out = torch.empty(p.out_elems, dtype=torch.float32, device="cuda")
    z = p.contract(out, want_z=True)
    torch.cuda.synchronize()
    d = p.describe()
    if prec == "auto":
        assert [s_["class"] for s_ in d["steps"]] == ["tcgen05"] * 3
    idx = sample(30, 256, 9)
    z_or = oracle.total_mass(net)
    want = oracle.recon_states(net, idx) / z_or
    got = out[torch.tensor(idx, device="cuda")].double().cpu().numpy()
    err = np.abs(got - want)
    print(f"grid30/{prec}: tiles {[s_['tile'] for s_ in d['steps']]} max|err| {err.max():.3e} "
          f"max|P| {np.abs(want).max():.3e} Z {z:.12f} (oracle {z_or:.12f})")
    assert abs(z - z_or) <= 1e-9
    assert err.max() <= FP32_ATOL
    assert err.max() <= 1e-4 * np.abs(want).max()
    p.close()
    h.close()
