"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: the FP32 and split-BF16 forms <= 1e-5 absolute per probability
(and 1e-4 of the largest); TF32 <= 1e-3 total variation; plain BF16, which
misses that gate, only within the bound of its arithmetic (check_tc).  Both are also
checked relative to the largest probability, since probabilities are ~2^-n.
All sizes are powers of two (dimension 2 outputs, dimension 4 cuts), so the
"ragged" cases are tiles wider than the operand (M, N or K below the tile),
odd qubit counts per subcircuit, a single state (F = 0), a single subcircuit,
zero cuts, and slicing."""
import functools

import numpy as np
import pytest

import oracle
from gen import Network, Node, tensors, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2502_03445_gb300 import tqc  # noqa: E402

FP32_ATOL = 1e-5
TC_TV = 1e-3


def run(net, out_f64=False, **kw):
    h = tqc.Network(net)
    p = tqc.Plan(h, **kw)
    out = torch.empty(p.out_elems, dtype=torch.float64 if out_f64 else torch.float32, device="cuda")
    z = p.contract(out, want_z=True)
    torch.cuda.synchronize()
    res = out.cpu().numpy().astype(np.float64)
    d = p.describe()
    p.close()
    h.close()
    return res, z, d


def check_fp32(got, want, z=1.0):
    err = np.abs(got - want / z)
    assert err.max() <= FP32_ATOL, err.max()
    # FP32 arithmetic: far tighter than the absolute gate, relative to the peak
    assert err.max() <= 1e-4 * max(np.abs(want / z).max(), 1e-30), (err.max(), np.abs(want).max())


def check_tv(got, want, z=1.0, tv=TC_TV):
    ref = want / z
    t = 0.5 * np.abs(got - ref).sum() / max(np.abs(ref).sum(), 1e-300)
    assert t <= tv, t


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def test_line10_plain_fp32():
    net, _ = workloads.line10()
    got, z, d = run(net, precision="fp32")
    want = oracle.recon_bin(net)
    assert abs(z - 1.0) < 1e-12
    check_fp32(got, want)


@pytest.mark.parametrize("seed,n,depth,n_sub", [(1, 7, 3, 3), (2, 9, 4, 3), (3, 10, 3, 4), (4, 12, 3, 4)])
def test_exact_circuits_fp32(seed, n, depth, n_sub):
    net, _ = workloads.small_exact(seed, n=n, depth=depth, n_sub=n_sub, max_cuts=8)
    got, z, _ = run(net, precision="fp32")
    check_fp32(got, oracle.recon_bin(net))


def small_pp(seed, n=14, m=4, cuts=7, w=9):
    return tensors.shape_matched_network(n, m, cuts, w, seed=seed)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("planner", [tqc.PLANNER_GREEDY, tqc.PLANNER_EXHAUSTIVE])
def test_pseudo_physical_fp32(seed, planner):
    net = small_pp(500 + seed, m=3 + seed % 3)
    got, z, _ = run(net, precision="fp32", planner=planner)
    assert abs(z - 1.0) < 1e-9
    check_fp32(got, oracle.recon_bin(net))


def all_orders(m):
    """Every SSA contraction order of m leaves (small m)."""
    out = []

    def rec(avail, nxt, acc):
        if len(avail) == 1:
            out.append(list(acc))
            return
        for i in range(len(avail)):
            for j in range(i + 1, len(avail)):
                rest = [x for k, x in enumerate(avail) if k not in (i, j)]
                rec(rest + [nxt], nxt + 1, acc + [[avail[i], avail[j]]])

    rec(list(range(m)), m, [])
    return out


def test_order_invariance():
    """Any contraction order gives the same result (§III-E-1)."""
    net = tensors.random_data_network(small_pp(601, n=12, m=4, cuts=6), 601)
    want = oracle.recon_bin(net)
    z_or = oracle.total_mass(net)
    orders = all_orders(4)
    assert len(orders) == 18
    for od in orders[::3]:
        got, z, _ = run(net, precision="fp32", order=od, flags=tqc.FLAG_NO_RENORM)
        assert abs(z - z_or) <= 1e-9 * abs(z_or)
        np.testing.assert_allclose(got, want, atol=1e-5 * np.abs(want).max(), rtol=0)


def test_slicing_matches_unsliced():
    """Slicing = a sum of smaller networks, summed in FP64 (§III-E-2)."""
    net = small_pp(602, n=14, m=4, cuts=8)
    want = oracle.recon_bin(net)
    for sliced in ([0], [2, 5], [1, 3, 6]):
        got, z, d = run(net, precision="fp32", sliced=sliced)
        assert d["sliced"] == sorted(sliced)
        check_fp32(got, want)
    got64, _, _ = run(net, precision="fp32", sliced=[4], out_f64=True)
    check_fp32(got64, want)


def test_budget_slicing():
    net = small_pp(603, n=14, m=4, cuts=8)
    h = tqc.Network(net, shape_only=True)
    ws = tqc.Plan(h, precision="fp32").describe()["ws_bytes"]
    h.close()
    got, _, d = run(net, precision="fp32", mem_budget=ws // 2)
    assert d["sliced"]
    check_fp32(got, oracle.recon_bin(net))


@pytest.mark.parametrize("seed", range(3))
def test_bins_and_fixed_bits(seed):
    net = small_pp(700 + seed, n=15, m=4, cuts=7)
    rng = np.random.Generator(np.random.PCG64(seed))
    free = sorted(rng.choice(15, size=9, replace=False).tolist())
    fixed = rng.integers(0, 2, size=15).astype(np.uint8)
    got, _, _ = run(net, precision="fp32", free_qubits=free, fixed_bits=fixed)
    check_fp32(got, oracle.recon_bin(net, free, fixed))
    # new fixed bits at contract time, same plan
    h = tqc.Network(net)
    p = tqc.Plan(h, precision="fp32", free_qubits=free, fixed_bits=fixed)
    out = torch.empty(p.out_elems, dtype=torch.float32, device="cuda")
    for r in range(2):
        fb = rng.integers(0, 2, size=15).astype(np.uint8)
        p.contract(out, fixed_bits=fb)
        check_fp32(out.cpu().numpy().astype(np.float64), oracle.recon_bin(net, free, fb))
    p.close()
    h.close()


def test_single_state_bin():
    net = small_pp(710, n=12, m=3, cuts=5)
    fixed = np.array([1, 0, 1, 1, 0, 0, 1, 0, 1, 1, 0, 1], np.uint8)
    got, _, _ = run(net, precision="fp32", free_qubits=[], fixed_bits=fixed)
    want = oracle.recon_bin(net, [], fixed)
    assert got.shape == (1,)
    check_fp32(got, want)


def test_single_subcircuit_and_zero_cuts():
    rng = np.random.Generator(np.random.PCG64(3))
    one = Network(6, 0, [Node([3, 0, 5, 1, 4, 2], [], [], rng.random(64))])
    got, z, _ = run(one, precision="fp32")
    check_fp32(got, oracle.recon_bin(one), oracle.total_mass(one))
    two = Network(7, 0, [Node([0, 4, 2], [], [], rng.random(8)), Node([6, 1, 3, 5], [], [], rng.random(16))])
    got, z, _ = run(two, precision="fp32", out_f64=True)
    check_fp32(got, oracle.recon_bin(two), oracle.total_mass(two))


def test_f32_input_tensors():
    net = small_pp(720, n=13, m=3, cuts=6)
    h = tqc.Network(net, dtype=tqc.F32)
    p = tqc.Plan(h, precision="fp32")
    out = torch.empty(p.out_elems, dtype=torch.float32, device="cuda")
    p.contract(out)
    got = out.cpu().numpy().astype(np.float64)
    want = oracle.recon_bin(net.astype(np.float32).astype(np.float64))
    check_fp32(got, want)


def test_contract_host_end_to_end():
    net = small_pp(730, n=13, m=4, cuts=6)
    h = tqc.Network(net)
    p = tqc.Plan(h, precision="fp32")
    host_out = np.empty(p.out_elems, np.float32)
    # new tensors from the host: a different seed, same shape
    net2 = tensors.pseudo_physical_network(13, net.meta["edges"], [nd.out_qubits for nd in net.nodes], 99)
    z = p.contract_host([nd.data for nd in net2.nodes], host_out)
    check_fp32(host_out.astype(np.float64), oracle.recon_bin(net2))
    assert abs(z - 1) < 1e-9


# ---------------------------------------------------------------- tensor-core forms
def two_node(seed, fa, fb, n_cuts, low_from_a, pseudo=True):
    """Two subcircuits, one step: M = 2^fa, N = 2^fb, K = 4^n_cuts.  Qubit 0
    belongs to the rows (A) or to the columns (B), which selects the
    epilogue's staging orientation."""
    n = fa + fb
    qa = list(range(fa)) if low_from_a else list(range(fb, n))
    qb = [q for q in range(n) if q not in qa]
    if fa < fb:   # the planner puts the larger operand on the rows
        pass
    edges = [(0, 1)] * n_cuts
    return tensors.pseudo_physical_network(n, edges, [qa, qb], seed) if pseudo else \
        tensors.random_data_network(tensors.pseudo_physical_network(n, edges, [qa, qb], seed), seed)


TC_CASES = [  # (fa, fb, cuts, qubit 0 on rows)
    (9, 7, 3, False), (9, 7, 3, True), (12, 8, 4, False), (10, 6, 3, True),
    (10, 4, 5, False), (10, 4, 3, True), (8, 8, 4, True), (11, 9, 3, False), (7, 7, 5, True),
]


@pytest.mark.parametrize("fa,fb,cuts,low_a", TC_CASES)
def test_tensor_core_step_bf16x3(fa, fb, cuts, low_a):
    net = two_node(800 + fa * 7 + cuts, fa, fb, cuts, low_a)
    got, z, d = run(net, precision="bf16x3")
    assert d["steps"][0]["class"] == "tcgen05", d["steps"]
    check_fp32(got, oracle.recon_bin(net))


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("fa,fb,cuts,low_a", TC_CASES[:5])
def test_tensor_core_step_bf16_tf32(prec, fa, fb, cuts, low_a):
    net = two_node(900 + fa * 7 + cuts, fa, fb, cuts, low_a)
    got, z, d = run(net, precision=prec)
    assert d["steps"][0]["class"] == "tcgen05"
    check_tc(prec, got, net, d)


# Deep-K steps (K = 4^6, 4^7): the default tile is the direct-epilogue form,
# 128 x 256 when N >= 256, 128 x 128 for split BF16 when N = 128.
UMMA_128x128, UMMA_128x64, UMMA_128x128_DEEP, UMMA_128x256_DEEP = 0, 1, 2, 3
DEEP_CASES = [  # (fa, fb, cuts, qubit 0 on rows)
    (8, 8, 6, True), (9, 8, 6, False), (9, 7, 6, True), (7, 8, 7, False),
]


def expected_deep_tile(d, prec):
    st = d["steps"][-1]
    if st["log2_n"] >= 8:
        return UMMA_128x256_DEEP
    return UMMA_128x128_DEEP if prec == "bf16x3" else UMMA_128x128


@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "tf32"])
@pytest.mark.parametrize("fa,fb,cuts,low_a", DEEP_CASES)
def test_tensor_core_deep_k(prec, fa, fb, cuts, low_a):
    net = two_node(1300 + fa * 7 + cuts, fa, fb, cuts, low_a)
    got, z, d = run(net, precision=prec)
    st = d["steps"][-1]
    assert st["class"] == "tcgen05" and st["log2_k"] == 2 * cuts
    assert st["tile"] == expected_deep_tile(d, prec), st
    want = oracle.recon_bin(net)
    if prec == "bf16x3":
        check_fp32(got, want)
    else:
        check_tc(prec, got, net, d, want)


def test_tensor_core_deep_k_sliced_f64():
    """Deep-K final step accumulating slices into the FP64 sum."""
    net = two_node(1400, 8, 8, 7, True)
    want = oracle.recon_bin(net)
    got, z, d = run(net, precision="bf16x3", sliced=[2], out_f64=True)
    assert d["sliced"] == [2] and d["steps"][-1]["tile"] == UMMA_128x256_DEEP
    check_fp32(got, want)


# K split of the final step: a deep-K step with fewer tiles than SMs runs
# its K loop in ranges on separate CTAs; the FP32 partials are summed in
# FP64 and stored in the step's own output mode (scaled FP32 or FP64, or the
# FP64 slice sum when sliced).
KSPLIT_CASES = [  # (fa, fb, cuts, form); N = 2^8: 128 x 256 tiles in every precision
    (8, 8, 6, "f32"), (8, 8, 7, "f32"), (9, 8, 7, "f64"), (8, 8, 7, "sliced"), (8, 9, 7, "sliced"),
]


@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "tf32"])
@pytest.mark.parametrize("fa,fb,cuts,form", KSPLIT_CASES)
def test_final_step_k_split(prec, fa, fb, cuts, form):
    net = two_node(1600 + fa * 7 + fb + cuts, fa, fb, cuts, True)
    want = oracle.recon_bin(net)
    kw = {"sliced": [2]} if form == "sliced" else {}
    got, z, d = run(net, out_f64=form != "f32", precision=prec, **kw)
    st = d["steps"][-1]
    assert st["tile"] == UMMA_128x256_DEEP and st["ksplit"] > 1, st
    assert d["sliced"] == ([2] if form == "sliced" else [])
    if prec == "bf16x3":
        check_fp32(got, want)
    else:
        check_tc(prec, got, net, d, want)


# K-blocked operands: tensor-core operands with rows longer than 64 KB are
# stored as [K / 64][rows][64] and copied with 3-D boxes.  Leaves get the
# layout from the ingest, an intermediate from its producing step.
def kblk_three_node(seed):
    outs = [list(range(0, 8)), list(range(8, 12)), list(range(12, 15))]
    return tensors.pseudo_physical_network(15, [(0, 1)] * 8 + [(1, 2)], outs, seed)


@functools.lru_cache(maxsize=2)
def kblk_three_node_oracle(seed):
    return oracle.recon_bin(kblk_three_node(seed))


@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "tf32"])
def test_k_blocked_operands(prec):
    """M = N = 128: the direct 128 x 128 form with a K split (split BF16)
    and the staged 128 x 128 form (BF16, TF32)."""
    net = two_node(1700, 7, 7, 8, True)
    want = oracle.recon_bin(net)
    got, z, d = run(net, precision=prec)
    st = d["steps"][-1]
    assert st["class"] == "tcgen05" and st["log2_k"] == 16 and st["kblk"] == 1, st
    if prec == "bf16x3":
        check_fp32(got, want)
    else:
        check_tc(prec, got, net, d, want)


@pytest.mark.parametrize("order", [[[1, 2], [0, 3]], [[0, 1], [3, 2]]])
@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
def test_k_blocked_intermediate_and_leaves(order, prec):
    """Order 1: a CUDA-core step writes the K-blocked operand of a deep
    tensor-core final step.  Order 2: the ingest writes K-blocked leaves for a
    128 x 64 tensor-core first step."""
    net = kblk_three_node(1710)
    want = kblk_three_node_oracle(1710)
    got, z, d = run(net, precision=prec, order=order)
    kst = [st for st in d["steps"] if st["kblk"]]
    assert len(kst) == 1 and kst[0]["log2_k"] == 16 and kst[0]["class"] == "tcgen05", d["steps"]
    if prec == "bf16x3":
        # 4^9 terms per probability with heavy cancellation (probabilities of
        # either sign): the FP32 gate holds, and the total
        # variation stays within the split-BF16 bound (operands exact to
        # about 2^-16, so 2^-15 per step on the absolute terms)
        assert np.abs(got - want).max() <= FP32_ATOL
        check_tv(got, want, tv=len(d["steps"]) * 2.0 ** -15 * abs_mass(net))
    else:
        check_tc(prec, got, net, d, want)


def kron_final_network(seed, cuts, fb=8):
    """Two nodes whose final step writes the bin in qubit order with a
    column qubit at bit 0 and seven row qubits above it: the direct
    epilogue's warp stores fill whole sectors, so a direct tile (128 x 256,
    or 128 x 128 when N = 128) is the default even at small K."""
    outs = [[1, 2, 3, 4, 5, 6, 7, 9, 11], [0, 8, 10, 12, 13, 14, 15, 16]]
    if fb == 7:
        outs = [[1, 2, 3, 4, 5, 6, 7, 9, 11, 16], [0, 8, 10, 12, 13, 14, 15]]
    return tensors.pseudo_physical_network(17, [(0, 1)] * cuts, outs, seed)


@pytest.mark.parametrize("fb", [8, 7])
@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "tf32"])
def test_final_step_direct_epilogue(prec, fb):
    net = kron_final_network(1500 + fb, 3, fb)
    want = oracle.recon_bin(net)
    got, z, d = run(net, precision=prec)
    st = d["steps"][-1]
    assert st["log2_n"] == fb and st["log2_k"] == 6, st
    assert st["tile"] == (UMMA_128x256_DEEP if fb == 8 else UMMA_128x128_DEEP), st
    if prec == "bf16x3":
        check_fp32(got, want)
    else:
        check_tc(prec, got, net, d, want)


def test_final_step_direct_epilogue_sliced_and_f64():
    net = kron_final_network(1501, 4)
    want = oracle.recon_bin(net)
    got, z, d = run(net, precision="bf16x3", sliced=[1], out_f64=True)       # FP64 slice sum
    assert d["sliced"] == [1] and d["steps"][-1]["tile"] == UMMA_128x256_DEEP
    check_fp32(got, want)
    got, z, d = run(net, precision="bf16x3", out_f64=True)                    # scaled FP64 output
    assert d["steps"][-1]["tile"] == UMMA_128x256_DEEP
    check_fp32(got, want)


def abs_mass(net):
    """sum_x of the reconstruction with |T_j| in place of T_j: the sum of
    the absolute values of every term, which bounds rounding errors."""
    a = Network(net.n_qubits, net.n_cuts,
                [Node(nd.out_qubits, nd.cut_ids, nd.cut_role, np.abs(nd.data)) for nd in net.nodes])
    return float(oracle.total_mass(a))


def check_tc(prec, got, net, d, want=None):
    """TF32 must meet the 1e-3 total-variation gate of the tensor-core
    forms.  Plain BF16 does NOT meet that gate on these pseudo-physical
    inputs (it lands near 1.2e-3 to 1.6e-3; include/tqc.h says so and the
    automatic choice never takes it), so it is tested only as what it is: a
    form whose error stays within the bound its arithmetic gives.  Every
    step rounds its two operands to 8 significant bits (unit roundoff
    2^-8), so each term of each probability carries a relative error below
    2 * n_steps * 2^-8 and TV <= n_steps * 2^-8 * sum_x sum_e |terms|."""
    if want is None:
        want = oracle.recon_bin(net)
    if prec == "tf32":
        check_tv(got, want)
        return
    bound = len(d["steps"]) * 2.0 ** -8 * abs_mass(net)
    check_tv(got, want, tv=bound)


def chain3(seed, variant, extra=0):
    """Three subcircuits A-B-C with three cuts on each link (K = 64 in both
    steps) and 16 qubits: both steps run on tensor cores, the first one
    writing the operand of the second.  The oracle sums 4^(6+extra) terms per
    state."""
    outs = [[0, 3, 6, 9, 12, 15], [1, 4, 7, 10, 13], [2, 5, 8, 11, 14]]
    if variant % 2:
        outs = [outs[1], outs[0], outs[2]]
    edges = [(0, 1)] * 3 + [(1, 2)] * 3 + [(0, 2)] * extra
    return tensors.pseudo_physical_network(16, edges, outs, seed)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "tf32"])
@pytest.mark.parametrize("seed", range(2))
def test_tensor_core_multi_step(prec, seed):
    """Networks whose intermediate steps run on tensor cores, so epilogues
    write BF16 / split-BF16 / TF32 operands for the next step."""
    net = chain3(1100 + seed, seed)
    got, z, d = run(net, precision=prec)
    classes = [s["class"] for s in d["steps"]]
    assert "tcgen05" in classes, d["steps"]
    want = oracle.recon_bin(net)
    if prec == "bf16x3":
        check_fp32(got, want)
    else:
        check_tc(prec, got, net, d, want)


def test_tensor_core_sliced():
    net = chain3(1200, 1, extra=1)
    want = oracle.recon_bin(net)
    got, z, d = run(net, precision="bf16x3", sliced=[1, 6])
    assert d["sliced"] == [1, 6]
    check_fp32(got, want)


def test_total_mass_tracks_uploads():
    """Z is cached per plan and recomputed after new tensors arrive."""
    base = small_pp(740, n=12, m=3, cuts=5)
    nets = [tensors.random_data_network(base, s) for s in (1, 2)]
    h = tqc.Network(nets[0])
    p = tqc.Plan(h, precision="fp32")
    out = torch.empty(p.out_elems, dtype=torch.float32, device="cuda")
    for rep, net in enumerate([nets[0], nets[0], nets[1], nets[1]]):
        if rep == 2:
            for j, nd in enumerate(net.nodes):
                h.upload(j, nd.data)
        z = p.contract(out, want_z=True)
        z_or = oracle.total_mass(net)
        assert abs(z - z_or) <= 1e-9 * abs(z_or), (rep, z, z_or)
        check_fp32(out.cpu().numpy().astype(np.float64), oracle.recon_bin(net), z_or)
    p.close()
    h.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_autotuned_plan_matches(prec):
    """The autotuner only changes tile shapes, never results."""
    net = chain3(1300, 0) if prec == "bf16x3" else small_pp(750, n=16, m=4, cuts=7)
    want = oracle.recon_bin(net)
    got, z, d = run(net, precision=prec, autotune=1)
    h = tqc.Network(net)
    p = tqc.Plan(h, precision=prec, autotune=1)
    out = torch.empty(p.out_elems, dtype=torch.float32, device="cuda")
    p.contract(out)
    d = p.describe()
    assert d["tuned"] == 1
    check_fp32(out.cpu().numpy().astype(np.float64), want)
    p.close()
    h.close()


def test_step_timeout_is_reported_once():
    """A tensor-core step whose bounded wait gives up (test hook) sets the
    plan's error word; a call with z_out reports it as TQC_ERR_TIMEOUT and
    clears it, so the next call is clean and correct."""
    net = chain3(1250, 0)
    want = oracle.recon_bin(net) / oracle.total_mass(net)
    h = tqc.Network(net)
    p = tqc.Plan(h, precision="bf16x3")
    assert "tcgen05" in [s_["class"] for s_ in p.describe()["steps"]]
    out = torch.empty(p.out_elems, dtype=torch.float32, device="cuda")
    p.contract(out)
    tqc.step_inject_stall(True)
    try:
        p.contract(out)                       # z_out NULL: nothing reported yet
    finally:
        tqc.step_inject_stall(False)
    torch.cuda.synchronize()
    with pytest.raises(tqc.TqcError) as ei:
        p.contract(out, want_z=True)          # reports the earlier call's timeout
    assert ei.value.status == tqc.ERR_TIMEOUT
    p.contract(out, want_z=True)              # cleared: clean
    check_fp32(out.cpu().numpy().astype(np.float64), want)
    p.close()
    h.close()
