"""Reuse of intermediates across bins (with TQC_FLAG_REUSE, tqc_contract keeps the previous call's
leaf operands and intermediates when only some subcircuits' fixed bits
change).  Every bin of a stream is checked against oracle C (the whole bin
by FP64 pairwise contraction) at the FP32 gate, with what each call kept
read from tqc_plan_describe."""
import itertools

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


ORDER = [[0, 1], [4, 2], [5, 3]]    # ((A B) C) D: D enters in the last step


OUTS = [[0, 4, 8, 12, 16], [1, 5, 9, 13, 17], [2, 6, 10, 14], [3, 7, 11, 15]]
EDGES = [(0, 1)] * 3 + [(1, 2)] * 3 + [(2, 3)] * 3     # K = 64 per link: tensor-core steps


def chain(seed):
    """Four subcircuits in a chain A-B-C-D, 18 qubits, 9 cuts."""
    return tensors.pseudo_physical_network(18, EDGES, OUTS, seed)


def check(out, net, free, fixed):
    want = oracle.recon_bin_pairwise(net, free, fixed) / oracle.total_mass(net)
    err = np.abs(out.cpu().numpy().astype(np.float64) - want).max()
    assert err <= FP32_ATOL and err <= 1e-4 * np.abs(want).max(), err


@pytest.mark.parametrize("precision", ["bf16x3", "fp32"])
def test_stream_over_one_subcircuits_fixed_bits(precision):
    net = chain(5100)
    h = tqc.Network(net)
    fixed_q = net.nodes[3].out_qubits[:3]
    free = [q for q in range(18) if q not in fixed_q]
    p = tqc.Plan(h, precision=precision, free_qubits=free, order=ORDER, flags=tqc.FLAG_REUSE)
    out = torch.empty(p.out_elems, dtype=torch.float32, device="cuda")
    n_steps = len(p.describe()["steps"])
    for k, bits in enumerate(itertools.product([0, 1], repeat=3)):
        fixed = np.zeros(18, np.uint8)
        fixed[fixed_q] = bits
        p.contract(out, fixed_bits=fixed)
        torch.cuda.synchronize()
        d = p.describe()
        if k:
            # every other leaf and every step before D's is kept
            assert d["reused_leaves"] == 3 and d["reused_steps"] == n_steps - 1, d
        check(out, net, free, fixed)
    p.close()
    h.close()


def test_invalidation():
    """New tensors, a first-contracted subcircuit's bits and the per-state
    path give correct results; without TQC_FLAG_REUSE nothing is kept."""
    net = chain(5200)
    free = list(range(14))
    h = tqc.Network(net)
    p = tqc.Plan(h, precision="bf16x3", free_qubits=free, flags=tqc.FLAG_REUSE)
    out = torch.empty(p.out_elems, dtype=torch.float32, device="cuda")
    fixed = np.zeros(18, np.uint8)
    p.contract(out, fixed_bits=fixed)
    check(out, net, free, fixed)
    # new tensors: nothing kept
    net2 = tensors.pseudo_physical_network(18, EDGES, OUTS, 5201)
    for jj, nd in enumerate(net2.nodes):
        h.upload(jj, nd.data)
    p.contract(out, fixed_bits=fixed)
    torch.cuda.synchronize()
    assert p.describe()["reused_steps"] == 0 and p.describe()["reused_leaves"] == 0
    check(out, net2, free, fixed)
    # every fixed qubit flipped (14..17 span several subcircuits)
    fixed[14:] = 1
    p.contract(out, fixed_bits=fixed)
    check(out, net2, free, fixed)
    # a single-state plan on the same network runs per state or fused; this
    # plan's workspace is untouched by the fused form and rewritten by the
    # per-state form, which clears what it kept
    ps = tqc.Plan(h, free_qubits=[])
    st = np.arange(5, dtype=np.uint64) * 12345
    ps.contract_states(st, torch.empty(5, dtype=torch.float32, device="cuda"))
    ps.close()
    p.contract(out, fixed_bits=fixed)
    check(out, net2, free, fixed)
    p.close()
    q = tqc.Plan(h, precision="bf16x3", free_qubits=free)      # without TQC_FLAG_REUSE
    for _ in range(2):
        q.contract(out, fixed_bits=fixed)
        assert q.describe()["reused_steps"] == 0
    check(out, net2, free, fixed)
    q.close()
    h.close()


def test_sliced_plan_keeps_only_slice_independent_tensors():
    net = chain(5300)
    free = list(range(15))
    h = tqc.Network(net)
    p = tqc.Plan(h, precision="bf16x3", free_qubits=free, sliced=[7], flags=tqc.FLAG_REUSE)
    out = torch.empty(p.out_elems, dtype=torch.float32, device="cuda")
    for bits in ([0, 0, 0], [1, 0, 1], [1, 1, 1]):
        fixed = np.zeros(18, np.uint8)
        fixed[15:] = bits
        p.contract(out, fixed_bits=fixed)
        torch.cuda.synchronize()
        check(out, net, free, fixed)
    p.close()
    h.close()
