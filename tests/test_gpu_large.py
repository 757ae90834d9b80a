"""Full-size workloads, checked through the C ABI against the FP64 oracles.

* 48-qubit QAOA p=1 (3-regular graph, 5 subcircuits of width <= 16, 16-24
  cuts), one bin of 2^24 states, contracted with the memory budget forcing
  slicing: the final step is a tensor-core GEMM with K = 4^9..4^11.
* The 64-qubit grid shape (6 subcircuits, width <= 20, 27 cuts), a stream of
  bins of 2^24 states: one plan, new node tensors uploaded per bin.
* The bench workload itself: the 30-qubit grid shape, the full 2^30 bin, in
  the launch configuration bench.py times -- every one of the 2^30 outputs
  against oracle C, in four chunks of 2^28.

No oracle produces a whole 2^24 bin of the tensor-bound networks in
reasonable time, so those tests check element by element

  (i) a sub-bin: the 2^k states that share random bits on all but k
      randomly chosen free qubits (1024 states for QAOA-48, 256 per grid64
      bin), computed at once by oracle C (whole-bin FP64 pairwise
      contraction);
  (ii) the 64 states of largest |P| on the device and 64 (QAOA-48) or 16
      (grid64) uniformly drawn states, each by oracle B (per-state
      elimination) in spawned processes;

plus properties that hold at any size: the bin's total mass Z (FP64 on the
device) against the oracle's, and the sum of all 2^24 outputs against Z.

Gates.  Every output of a form meets the FP32 gate of 1e-5 absolute per
probability.  Forms whose steps all run in FP32 or split BF16 also meet a
per-state bound against the scale of the terms, s = sum over the bin of the
reconstruction with |T_j| in place of T_j, divided by 2^F: probabilities of
pseudo-physical networks are signed sums whose terms cancel, so |P| alone
says nothing about the rounding error.  Bound: n_steps * 2^-12 * s (each step
rounds its products to about 2^-16 relative in split BF16, 2^-24 in FP32,
and accumulates K terms in FP32 whose randomly signed rounding errors grow
like sqrt(K) * 2^-24 <= 2^-13 for K <= 2^22).  A plan with a TF32 step is
held to the 1e-3 total-variation gate of the tensor-core forms instead,
measured over the checked states: sum |dP| / sum |P|."""
import functools

import numpy as np
import pytest

import oracle
from gen import Network, Node, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2502_03445_gb300 import tqc  # noqa: E402

FP32_ATOL = 1e-5
TC_TV = 1e-3
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


def sub_bin(net, k, seed):
    """(entry indices into the full bin, oracle C values) of the sub-bin
    whose k free qubits are drawn at random and whose other qubits carry
    random bits."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = net.n_qubits
    free = sorted(int(q) for q in rng.choice(n, size=k, replace=False))
    fixed = rng.integers(0, 2, size=n).astype(np.uint8)
    idx = oracle.bin_states(n, free, fixed, np.arange(1 << k))
    return np.array(idx, dtype=np.int64), oracle.recon_bin_pairwise(net, free, fixed)


def check_result(net, spec, got, z, d, k_sub, seed, n_top, n_uni, label):
    """got: raw (unnormalised) FP64 copy of the device output of the bin
    whose qubits are all free (entry index = state)."""
    z_or = oracle.total_mass(net)
    s = abs_scale(net)
    n_steps = len(d["steps"])
    tf32 = any(st["class"] == "tcgen05" and st["prec"] == "tf32" for st in d["steps"])
    # total mass: an FP64 scalar network on the device
    assert abs(z - z_or) <= 1e-9 * abs(z_or) + 1e-12 * s * (1 << net.n_qubits), (z, z_or)
    # the sum of every output equals Z (error: 2^F states x the per-state bound, but signed
    # rounding errors average out; the bound kept here is the per-state one x sqrt(2^F))
    tot = float(got.sum())
    tol_sum = n_steps * 2.0 ** -(10 if tf32 else 12) * s * np.sqrt(float(1 << net.n_qubits))
    assert abs(tot - z_or) <= tol_sum, (tot, z_or, tol_sum)
    # (i) a sub-bin by oracle C
    idx_c, want_c = sub_bin(net, k_sub, seed)
    # (ii) the largest |P| and uniformly drawn states by oracle B
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    top = np.argpartition(-np.abs(got), n_top)[:n_top]
    uni = rng.integers(0, 1 << net.n_qubits, size=n_uni)
    idx_b = np.unique(np.concatenate([top, uni]).astype(np.int64))
    want_b = oracle.recon_states_elim_pool(spec, idx_b.tolist())
    idx = np.concatenate([idx_c, idx_b])
    want = np.concatenate([want_c, want_b])
    err = np.abs(got[idx] - want)
    tv = 0.5 * err.sum() / np.abs(want).sum()
    print(f"{label}: slices={d.get('sliced')} steps={[(t['log2_m'], t['log2_n'], t['log2_k'], t['class'], t['prec']) for t in d['steps']]}"
          f" checked={len(idx)} (sub-bin {len(idx_c)}, oracle B {len(idx_b)}) Z={z:.6e} (oracle {z_or:.6e})"
          f" sum-Z={tot - z_or:.3e} max|err|={err.max():.3e} scale={s:.3e} err/scale={err.max() / s:.3e}"
          f" tv={tv:.3e} max|P|={np.abs(want).max():.3e}")
    assert err.max() <= FP32_ATOL
    if tf32:
        assert tv <= TC_TV, tv
    else:
        assert err.max() <= n_steps * 2.0 ** -12 * s, (err.max(), s)
    return tv


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
    check_result(net, ("gen.workloads", "qaoa48", (0,)), got, z, d, 10, 4, 64, 64, f"qaoa48/{prec}")
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
        check_result(net, ("gen.workloads", "grid64_bin", (0, b)), got, z, d, 8, 50 + b, 64, 16, f"grid64/bin{b}")
    p.close()
    h.close()


@pytest.mark.parametrize("prec", ["auto", "fp32"])
def test_grid30_full_vector(prec):
    """bench.py's workload and launch configuration: every qubit free, the
    default plan (tensor-core steps with the direct and staged epilogues, or
    the plain FP32 form), renormalised FP32 output.  Gates: 1e-5 absolute
    everywhere; 1e-4 of the largest probability for FP32-class forms, total
    variation 1e-3 when a step runs in TF32.  All 2^30 outputs are
    compared with oracle C, a quarter at a time (qubits 28 and 29 fixed), and
    256 uniformly drawn ones with oracle A."""
    net = workloads.grid30(0)
    h = tqc.Network(net)
    p = tqc.Plan(h, precision=prec)
    out = torch.empty(p.out_elems, dtype=torch.float32, device="cuda")
    z = p.contract(out, want_z=True)
    torch.cuda.synchronize()
    d = p.describe()
    tf32 = any(s_["class"] == "tcgen05" and s_["prec"] == "tf32" for s_ in d["steps"])
    if prec == "auto":
        assert d["steps"][-1]["class"] == "tcgen05" and d["steps"][-1]["prec"] == "bf16x3", d["steps"]
    z_or = oracle.total_mass(net)
    assert abs(z - z_or) <= 1e-9
    got = out.cpu().numpy()
    del out
    # oracle A on uniformly drawn states
    rng = np.random.Generator(np.random.PCG64(9))
    idx = sorted(set(int(i) for i in rng.integers(0, 1 << 30, size=256)))
    err_a = np.abs(got[idx].astype(np.float64) - oracle.recon_states(net, idx) / z_or).max()
    # oracle C on every output, in quarters
    max_err, max_p, abs_sum, err_sum = 0.0, 0.0, 0.0, 0.0
    for quarter in range(4):
        fixed = np.zeros(30, np.uint8)
        fixed[28], fixed[29] = quarter & 1, quarter >> 1
        want = oracle.recon_bin_pairwise(net, list(range(28)), fixed)
        want /= z_or
        part = got[quarter << 28:(quarter + 1) << 28].astype(np.float64)
        part -= want
        np.abs(part, out=part)
        max_err = max(max_err, float(part.max()))
        err_sum += float(part.sum())
        max_p = max(max_p, float(np.abs(want).max()))
        abs_sum += float(np.abs(want).sum())
        del want, part
    tv = 0.5 * err_sum / abs_sum
    print(f"grid30/{prec}: tiles {[s_['tile'] for s_ in d['steps']]} full vector: max|err| {max_err:.3e} "
          f"max|P| {max_p:.3e} (err/max {max_err / max_p:.2e}) TV {tv:.3e}; oracle A sample max|err| {err_a:.3e}")
    assert err_a <= FP32_ATOL and max_err <= FP32_ATOL
    if tf32:        # a TF32 step: the total-variation gate of the tensor-core forms
        assert tv <= TC_TV, tv
    else:           # FP32-class arithmetic: also within 1e-4 of the largest probability
        assert err_a <= 1e-4 * max_p and max_err <= 1e-4 * max_p
    p.close()
    h.close()
