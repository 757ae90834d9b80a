"""The allocation-free entry point (tqc_contract_noalloc).

It serves callers that cannot allocate device memory when they reconstruct
(an allocator owned by another framework, a capped MPS client, a loop that
must not synchronise the device).  It must give the oracle's results and the
same results as tqc_contract with every intermediate in the library's fixed
scratch array, call after call, allocate nothing, report a bounded device
wait that gave up, and refuse plans that need more scratch than the array
has.

This file is named to be collected last: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import oracle
from gen import tensors
from paper_2502_03445_gb300 import tqc

FP32_ATOL = 1e-5


def three_subcircuits(seed):
    outs = [[0, 3, 6, 9, 12, 15], [1, 4, 7, 10, 13], [2, 5, 8, 11, 14]]
    edges = [(0, 1)] * 3 + [(1, 2)] * 3
    return tensors.pseudo_physical_network(16, edges, outs, seed)


def check_fp32(got, want):
    err = np.abs(got - want).max()
    assert err <= FP32_ATOL, err
    assert err <= 1e-4 * np.abs(want).max(), (err, np.abs(want).max())


def cuda_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


def test_rejects_plans_beyond_the_scratch_array():
    from gen import workloads
    net = workloads.grid30()
    h = tqc.Network(net, shape_only=True)
    p = tqc.Plan(h, precision="bf16x3")
    dummy = (ctypes.c_void_p * 4)(*([16] * 4))
    st = tqc.lib().tqc_contract_noalloc(p.handle, ctypes.cast(dummy, ctypes.c_void_p), tqc.F64, None, 16,
                                        tqc.F32, None)
    assert st == tqc.ERR_UNSUPPORTED
    msg = tqc.lib().tqc_last_error().decode()
    assert "scratch" in msg and str(tqc.lib().tqc_noalloc_scratch_bytes()) in msg
    p.close()
    h.close()


@pytest.mark.gpu
@pytest.mark.parametrize("precision,sliced", [("bf16x3", None), ("fp32", [2])])
def test_matches_allocating_entry_point_twice(precision, sliced):
    torch = cuda_or_skip()
    net = three_subcircuits(4242)
    want = oracle.recon_bin(net) / oracle.total_mass(net)
    # the allocating entry point on a network with device copies
    h = tqc.Network(net)
    ref_plan = tqc.Plan(h, precision=precision, sliced=sliced)
    ref = torch.empty(ref_plan.out_elems, dtype=torch.float32, device="cuda")
    ref_plan.contract(ref)
    torch.cuda.synchronize()
    ref_np = ref.cpu().numpy().astype(np.float64)
    check_fp32(ref_np, want)
    # allocation-free: plan from a shape-only network, the caller's tensors
    hs = tqc.Network(net, shape_only=True)
    plan = tqc.Plan(hs, precision=precision, sliced=sliced)
    d_tensors = [torch.from_numpy(np.ascontiguousarray(nd.data)).cuda() for nd in net.nodes]
    for call in range(2):
        out = torch.full((plan.out_elems,), float("nan"), dtype=torch.float32, device="cuda")
        plan.contract_noalloc(d_tensors, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        check_fp32(got, want)
        err = np.abs(got - ref_np).max()
        assert err <= FP32_ATOL and err <= 1e-4 * np.abs(ref_np).max(), (call, err)
    plan.close()
    hs.close()
    ref_plan.close()
    h.close()


@pytest.mark.gpu
def test_f32_tensors_and_fixed_bits_match_the_oracle():
    """FP32 device tensors (in_dtype F32) and a bin with explicit fixed bits,
    given at plan time and overridden at call time."""
    torch = cuda_or_skip()
    net = three_subcircuits(4243)
    free = [0, 1, 2, 3, 5, 6, 8, 9, 10, 11, 12, 14]
    fixed = np.zeros(16, np.uint8)
    fixed[[4, 13]] = 1
    fixed2 = np.zeros(16, np.uint8)
    fixed2[[7, 15]] = 1
    hs = tqc.Network(net, shape_only=True)
    plan = tqc.Plan(hs, precision="bf16x3", free_qubits=free, fixed_bits=fixed)
    d32 = [torch.from_numpy(np.ascontiguousarray(nd.data, dtype=np.float32)).cuda() for nd in net.nodes]
    net32 = net.astype(np.float32).astype(np.float64)   # the values the device sees
    for fb in (None, fixed2):
        out = torch.full((plan.out_elems,), float("nan"), dtype=torch.float32, device="cuda")
        plan.contract_noalloc(d32, out, in_dtype=tqc.F32, fixed_bits=fb)
        torch.cuda.synchronize()
        want = oracle.recon_bin(net32, free, fixed if fb is None else fb) / oracle.total_mass(net32)
        check_fp32(out.cpu().numpy().astype(np.float64), want)
    plan.close()
    hs.close()


@pytest.mark.gpu
def test_allocates_nothing_and_leaves_the_plan_alone():
    """A plan that asks for the autotuner and per-step profiling: the call
    neither autotunes nor profiles nor prepares the plan's own workspace, and
    the device's free memory does not move across it."""
    torch = cuda_or_skip()
    net = three_subcircuits(4244)
    want = oracle.recon_bin(net) / oracle.total_mass(net)
    hs = tqc.Network(net, shape_only=True)
    plan = tqc.Plan(hs, precision="bf16x3", autotune=1)
    plan.profile(True)
    d_tensors = [torch.from_numpy(np.ascontiguousarray(nd.data)).cuda() for nd in net.nodes]
    out = torch.full((plan.out_elems,), float("nan"), dtype=torch.float32, device="cuda")
    plan.contract_noalloc(d_tensors, out)          # loads the modules the call uses
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        plan.contract_noalloc(d_tensors, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    d = plan.describe()
    assert d["ready"] == 0 and d["tuned"] == 0, d
    assert all(st["ksplit"] == 1 for st in d["steps"])
    assert plan.step_time(0)[1] == 0               # no profiling events were recorded
    check_fp32(out.cpu().numpy().astype(np.float64), want)
    plan.close()
    hs.close()


@pytest.mark.gpu
def test_ignores_autotune_and_k_split():
    """A plan that asks for the autotuner, on a network whose deep-K final
    step the allocating entry point splits along K: the allocation-free call
    does neither (both would allocate) and still gives the same result."""
    torch = cuda_or_skip()
    net = tensors.pseudo_physical_network(16, [(0, 1)] * 6, [list(range(8)), list(range(8, 16))], 4300)
    want = oracle.recon_bin(net) / oracle.total_mass(net)
    h = tqc.Network(net)
    ref_plan = tqc.Plan(h, precision="bf16x3")
    ref = torch.empty(ref_plan.out_elems, dtype=torch.float32, device="cuda")
    ref_plan.contract(ref)
    torch.cuda.synchronize()
    assert ref_plan.describe()["steps"][-1]["ksplit"] > 1
    ref_np = ref.cpu().numpy().astype(np.float64)
    hs = tqc.Network(net, shape_only=True)
    plan = tqc.Plan(hs, precision="bf16x3", autotune=1)
    d_tensors = [torch.from_numpy(np.ascontiguousarray(nd.data)).cuda() for nd in net.nodes]
    out = torch.full((plan.out_elems,), float("nan"), dtype=torch.float32, device="cuda")
    plan.contract_noalloc(d_tensors, out)
    torch.cuda.synchronize()
    d = plan.describe()
    assert d["tuned"] == 0 and all(st["ksplit"] == 1 for st in d["steps"]), d["steps"]
    got = out.cpu().numpy().astype(np.float64)
    check_fp32(got, want)
    err = np.abs(got - ref_np).max()
    assert err <= FP32_ATOL and err <= 1e-4 * np.abs(ref_np).max(), err
    plan.close()
    hs.close()
    ref_plan.close()
    h.close()


@pytest.mark.gpu
def test_reports_a_wait_that_gave_up():
    """With the step stall hook on, a tensor-core step's bounded wait gives
    up: the call returns TQC_ERR_TIMEOUT (it synchronises and reads its error
    word).  The next call, hook off, is clean and correct."""
    torch = cuda_or_skip()
    net = three_subcircuits(4245)
    want = oracle.recon_bin(net) / oracle.total_mass(net)
    hs = tqc.Network(net, shape_only=True)
    plan = tqc.Plan(hs, precision="bf16x3")
    assert "tcgen05" in [st["class"] for st in plan.describe()["steps"]]
    d_tensors = [torch.from_numpy(np.ascontiguousarray(nd.data)).cuda() for nd in net.nodes]
    out = torch.empty(plan.out_elems, dtype=torch.float32, device="cuda")
    tqc.step_inject_stall(True)
    try:
        with pytest.raises(tqc.TqcError) as ei:
            plan.contract_noalloc(d_tensors, out)
    finally:
        tqc.step_inject_stall(False)
    assert ei.value.status == tqc.ERR_TIMEOUT
    plan.contract_noalloc(d_tensors, out)
    torch.cuda.synchronize()
    check_fp32(out.cpu().numpy().astype(np.float64), want)
    plan.close()
    hs.close()
