"""The fused pair of tensor-core steps (fused.cu) against the oracle and the
unfused steps.

The fused kernel computes the first step's tile into tensor memory, splits
it into BF16 hi / lo planes exactly as the unfused epilogue does, lays it out
as the second step's operand in shared memory and runs the second step's
MMAs in the same order: its results must equal the unfused plan's bit for
bit.  Both are checked against oracle C (the whole bin by FP64 pairwise
contraction) at the FP32 gate."""
import numpy as np
import pytest

import oracle
from gen import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2502_03445_gb300 import tqc  # noqa: E402

FP32_ATOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def run(h, free, fixed, flags=0):
    p = tqc.Plan(h, free_qubits=free, fixed_bits=fixed, flags=flags)
    out = torch.empty(p.out_elems, dtype=torch.float32, device="cuda")
    p.contract(out, want_z=True)
    torch.cuda.synchronize()
    d = p.describe()
    p.close()
    return out.cpu().numpy(), d


@pytest.mark.parametrize("fixed_q,bits", [((21, 22, 24, 25, 27, 28, 29), (1, 0, 1, 1, 0, 0, 1)),
                                          ((25, 27, 28, 29), (0, 1, 1, 0)),
                                          ((27, 28, 29), (1, 1, 1))])
def test_grid30_bins_fused_equal_unfused_and_oracle(fixed_q, bits):
    net = workloads.grid30(0)
    free = [q for q in range(30) if q not in fixed_q]
    fixed = np.zeros(30, np.uint8)
    fixed[list(fixed_q)] = bits
    h = tqc.Network(net)
    got, d = run(h, free, fixed)
    assert [s["fuse"] for s in d["steps"]] == [1, 2, 0], d["steps"]
    ref, d0 = run(h, free, fixed, flags=tqc.FLAG_NO_FUSE)
    assert [s["fuse"] for s in d0["steps"]] == [0, 0, 0]
    h.close()
    np.testing.assert_array_equal(got, ref)
    want = oracle.recon_bin_pairwise(net, free, fixed) / oracle.total_mass(net)
    err = np.abs(got.astype(np.float64) - want)
    assert err.max() <= FP32_ATOL and err.max() <= 1e-4 * np.abs(want).max(), err.max()


def test_unaligned_bin_is_not_fused():
    net = workloads.grid30(0)
    h = tqc.Network(net, shape_only=True)
    p = tqc.Plan(h, free_qubits=list(range(4, 30)))
    assert all(s["fuse"] == 0 for s in p.describe()["steps"])
    p.close()
    h.close()


def test_fused_timeout_is_reported():
    """The stall hook reaches the fused kernel too: its bounded wait gives
    up, the call with z_out reports it, and the next call is clean."""
    net = workloads.grid30(0)
    free = [q for q in range(30) if q not in (21, 22, 24, 25, 27, 28, 29)]
    h = tqc.Network(net)
    p = tqc.Plan(h, free_qubits=free)
    assert p.describe()["steps"][0]["fuse"] == 1
    out = torch.empty(p.out_elems, dtype=torch.float32, device="cuda")
    p.contract(out)
    tqc.step_inject_stall(True)
    try:
        with pytest.raises(tqc.TqcError) as ei:
            p.contract(out, want_z=True)
    finally:
        tqc.step_inject_stall(False)
    assert ei.value.status == tqc.ERR_TIMEOUT
    p.contract(out, want_z=True)
    torch.cuda.synchronize()
    want = oracle.recon_bin_pairwise(net, free, np.zeros(30, np.uint8)) / oracle.total_mass(net)
    assert np.abs(out.cpu().numpy().astype(np.float64) - want).max() <= FP32_ATOL
    p.close()
    h.close()
