"""The allocation-free entry point (tqc_contract_noalloc).

It serves callers that cannot allocate device memory when they reconstruct
(an allocator owned by another framework, a capped MPS client, a loop that
must not synchronise the device).  It must give the same results as
tqc_contract with every intermediate in the library's fixed scratch array,
call after call, and refuse plans that need more scratch than the array has.

This file is named to be collected last: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from gen import tensors
from paper_2502_03445_gb300 import tqc

FP32_ATOL = 1e-5


def three_subcircuits(seed):
    outs = [[0, 3, 6, 9, 12, 15], [1, 4, 7, 10, 13], [2, 5, 8, 11, 14]]
    edges = [(0, 1)] * 3 + [(1, 2)] * 3
    return tensors.pseudo_physical_network(16, edges, outs, seed)


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
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    net = three_subcircuits(4242)
    # reference: the allocating entry point on a network with device copies
    h = tqc.Network(net)
    ref_plan = tqc.Plan(h, precision=precision, sliced=sliced)
    ref = torch.empty(ref_plan.out_elems, dtype=torch.float32, device="cuda")
    ref_plan.contract(ref)
    torch.cuda.synchronize()
    ref_np = ref.cpu().numpy().astype(np.float64)
    # allocation-free: plan from a shape-only network, the caller's tensors
    hs = tqc.Network(net, shape_only=True)
    plan = tqc.Plan(hs, precision=precision, sliced=sliced)
    d_tensors = [torch.from_numpy(np.ascontiguousarray(nd.data)).cuda() for nd in net.nodes]
    for call in range(2):
        out = torch.full((plan.out_elems,), float("nan"), dtype=torch.float32, device="cuda")
        plan.contract_noalloc(d_tensors, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        err = np.abs(got - ref_np).max()
        assert err <= FP32_ATOL, (call, err)
        assert err <= 1e-4 * np.abs(ref_np).max(), (call, err)
    plan.close()
    hs.close()
    ref_plan.close()
    h.close()


@pytest.mark.gpu
def test_ignores_autotune_and_k_split():
    """A plan that asks for the autotuner, on a network whose deep-K final
    step the allocating entry point splits along K: the allocation-free call
    does neither (both would allocate) and still gives the same result."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    net = tensors.pseudo_physical_network(16, [(0, 1)] * 6, [list(range(8)), list(range(8, 16))], 4300)
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
    err = np.abs(out.cpu().numpy().astype(np.float64) - ref_np).max()
    assert err <= FP32_ATOL and err <= 1e-4 * np.abs(ref_np).max(), err
    plan.close()
    hs.close()
    ref_plan.close()
    h.close()
