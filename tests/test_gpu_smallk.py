"""The small-K CUDA-core tile (smallk.cuh) against the general CUDA-core
tiles and the oracle.

Steps whose subcircuits share at most two cut edges (K = 1, 4 or 16) take a
tile shaped for the write-out.  It sums k in the same order with the same
fused multiply-adds as the general 64 x 64 .. 128 x 128 tiles, so the two
must agree bit for bit (TQC_FLAG_NO_SMALLK selects the general tiles); both
are checked against oracle C (the whole bin by FP64 pairwise contraction)
at the FP32 gate.  The cases cover K = 1, 4 and 16, tiles of 8 and more
columns (4 x 8 results per thread) and of 4 columns (8 x 4), direct stores
along rows and along columns, all four arrangements of the staged form's
16-byte chunks (rows 0-1, columns 0-1, row then column, column then row
lowest), a final step, intermediates written as FP32 and as split-BF16 /
TF32 operands of a tensor-core step, FP64 output, and the batched launch."""
import numpy as np
import pytest

import oracle
from gen import tensors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2502_03445_gb300 import tqc  # noqa: E402

FP32_ATOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _outs(n, groups):
    """Qubit lists of the subcircuits: `groups` is a list of (kind, count)
    with kind "hi" (the highest unused qubits), "lo" (the lowest), "even"
    (every other unused qubit from the lowest), "rest" (all unused) or
    "set" (count: an explicit list)."""
    free = list(range(n))
    res = []
    for kind, cnt in groups:
        if kind == "set":
            pick = list(cnt)
        elif kind == "lo":
            pick = free[:cnt]
        elif kind == "hi":
            pick = free[-cnt:]
        elif kind == "even":
            pick = free[0::2][:cnt]
        else:
            pick = free[:]
        res.append(sorted(pick))
        free = [q for q in free if q not in pick]
    assert not free
    return res


# name: (n_qubits, edges, subcircuit qubits, forced order or None, precision)
CASES = {
    # final step M = 2^16, N = 2^4, K = 16; column bits lowest (row-major staging, float4 gathers)
    "final_k16_narrow": (20, [(0, 1)] * 2, [("hi", 16), ("lo", 4)], None, "fp32"),
    # K = 4, interleaved row / column bits (paired or scalar gathers)
    "final_k4_interleaved": (18, [(0, 1)], [("even", 9), ("rest", 9)], None, "fp32"),
    # four columns: 8 x 4 results per thread; column-major staging
    "final_k16_four_columns": (16, [(0, 1)] * 2, [("lo", 14), ("hi", 2)], None, "fp32"),
    # K = 1 (an outer product of two subcircuits without a shared cut), then K = 16
    "outer_product_then_k16": (17, [(0, 1), (1, 2)], [("lo", 6), ("even", 5), ("hi", 6)],
                               [[0, 2], [3, 1]], "fp32"),
    # staged, the result's two lowest bits rows 0, 1 (row quads as float4 chunks)
    "final_k4_staged_rows_lowest": (18, [(0, 1)], [("set", [0, 1] + list(range(4, 12))), ("rest", 8)], None, "fp32"),
    # staged, column 0 then row 0 lowest (2 x 2 blocks as float4 chunks)
    "final_k16_staged_col_then_row": (17, [(0, 1)] * 2, [("set", [1] + list(range(4, 13))), ("rest", 7)], None,
                                      "fp32"),
    # a K = 16 intermediate feeding a tensor-core step (K = 64) as split-BF16 / TF32 operands
    "k16_into_tensor_core": (20, [(0, 1)] * 2 + [(1, 2)] * 3, [("hi", 8), ("even", 6), ("lo", 6)],
                             [[0, 1], [3, 2]], "auto"),
}


def network(name, seed):
    n, edges, groups, order, prec = CASES[name]
    return tensors.pseudo_physical_network(n, edges, _outs(n, groups), seed), order, prec


def run(h, net, order, prec, flags=0, out_dtype=torch.float32):
    p = tqc.Plan(h, precision=prec, order=order, flags=flags)
    out = torch.empty(p.out_elems, dtype=out_dtype, device="cuda")
    p.contract(out, want_z=True)
    torch.cuda.synchronize()
    d = p.describe()
    p.close()
    return out.cpu().numpy(), d


def check_oracle(got, net):
    want = oracle.recon_bin_pairwise(net) / oracle.total_mass(net)
    err = np.abs(got.astype(np.float64) - want)
    assert err.max() <= FP32_ATOL and err.max() <= 1e-4 * np.abs(want).max(), err.max()


@pytest.mark.parametrize("name", sorted(CASES))
def test_small_k_equals_general_tiles_and_oracle(name):
    net, order, prec = network(name, 6100 + sorted(CASES).index(name))
    h = tqc.Network(net)
    got, d = run(h, net, order, prec)
    small = [s for s in d["steps"] if s["class"] == "simt" and s["log2_k"] in (0, 2, 4)]
    assert small and all(s["tile"] == 3 for s in small), d["steps"]
    ref, d0 = run(h, net, order, prec, flags=tqc.FLAG_NO_SMALLK)
    assert all(s["tile"] != 3 for s in d0["steps"] if s["class"] == "simt")
    h.close()
    np.testing.assert_array_equal(got, ref)
    check_oracle(got, net)


def test_small_k_fp64_output():
    net, order, prec = network("final_k4_interleaved", 6200)
    h = tqc.Network(net)
    got, _ = run(h, net, order, prec, out_dtype=torch.float64)
    ref, _ = run(h, net, order, prec, flags=tqc.FLAG_NO_SMALLK, out_dtype=torch.float64)
    h.close()
    np.testing.assert_array_equal(got, ref)
    check_oracle(got, net)


def test_small_k_in_batched_launch():
    """The batch runs a plan's small-K steps with the same tile: its results
    equal the standalone contraction's bit for bit."""
    hs, plans, outs, refs, nets = [], [], [], [], []
    for k, name in enumerate(sorted(CASES)):
        net, order, _ = network(name, 6300 + k)
        h = tqc.Network(net)
        p = tqc.Plan(h, precision="fp32", order=order)
        o = torch.empty(p.out_elems, dtype=torch.float32, device="cuda")
        p.contract(o)
        torch.cuda.synchronize()
        assert any(s["tile"] == 3 for s in p.describe()["steps"])
        refs.append(o.cpu().numpy())
        hs.append(h)
        plans.append(p)
        outs.append(torch.full_like(o, float("nan")))
        nets.append(net)
    tqc.contract_batch(plans, outs)
    tqc.batch_status()
    for o, ref, net in zip(outs, refs, nets):
        got = o.cpu().numpy()
        np.testing.assert_array_equal(got, ref)
        check_oracle(got, net)
    for p in plans:
        p.close()
    for h in hs:
        h.close()
