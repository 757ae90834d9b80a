"""Heavy state selection on the GPU against its oracle (§IV, §VII-A).

* The device norms equal the oracle's (FP64; the FP32 upload against the
  oracle on the same rounded values).
* The selection equals the oracle's selection run on the device norms (the
  decision is taken on the same numbers); on networks without near ties it
  also equals the selection on the oracle's own norms.
* The selected network, contracted by the ordinary plan / contract path,
  gives every product state's probability (oracle A on the full states it
  stands for), and exact zeros on the padding entries.
* P_HSS on the paper's four circuit families against the oracle's."""
import math

import numpy as np
import pytest

import oracle
from gen import tensors, workloads
from oracle import hss

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2502_03445_gb300 import tqc  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def networks():
    out = [workloads.hss_circuit(f, 12)[0] for f in workloads.HSS_FAMILIES]
    out.append(tensors.shape_matched_network(14, 4, 7, 9, seed=4100))       # pseudo-physical, 4 subcircuits
    out.append(tensors.random_data_network(tensors.shape_matched_network(13, 3, 6, 8, seed=4101), 4101))
    return out


def device_norms(h, net):
    res = []
    for j, nd in enumerate(net.nodes):
        buf = torch.empty(1 << nd.n_out, dtype=torch.float64, device="cuda")
        h.hss_norms(j, buf)
        res.append(buf.cpu().numpy())
    return res


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("k", range(6))
def test_norms_match_oracle(k, dtype):
    net = networks()[k]
    if dtype == "f32":
        net = net.astype(np.float32).astype(np.float64)     # the values the device holds
    h = tqc.Network(net, dtype=tqc.F64 if dtype == "f64" else tqc.F32)
    got = device_norms(h, net)
    want = hss.state_norms(net)
    for g, w in zip(got, want):
        np.testing.assert_allclose(g, w, rtol=1e-12, atol=1e-300)
    h.close()


@pytest.mark.parametrize("k", range(6))
def test_norms_are_deterministic(k):
    """The norm sums split over cut assignments are added in a fixed order:
    repeated calls give bit-identical norms, so exact ties between states
    resolve the same way every time."""
    net = networks()[k]
    h = tqc.Network(net)
    first = device_norms(h, net)
    for _ in range(3):
        for a, b in zip(first, device_norms(h, net)):
            assert np.array_equal(a, b)
    h.close()


@pytest.mark.parametrize("k", range(6))
@pytest.mark.parametrize("s_max", [1, 5, 64, 1 << 30])
def test_selection_matches_oracle(k, s_max):
    net = networks()[k]
    h = tqc.Network(net)
    sel, n_states = h.hss_select(s_max)
    sel = [x.tolist() for x in sel]
    assert sel == hss.select(device_norms(h, net), s_max)
    assert n_states == math.prod(len(x) for x in sel)
    if k >= 4:   # random data: no ties, so the oracle's own norms decide the same
        assert sel == hss.select(hss.state_norms(net), s_max)
    h.close()


@pytest.mark.parametrize("prec", ["fp32", "auto"])
@pytest.mark.parametrize("k", range(6))
def test_selected_network_reconstructs_product_states(k, prec):
    net = networks()[k]
    h = tqc.Network(net)
    sel, _ = h.hss_select(48)
    sub = h.select(sel)
    p = tqc.Plan(sub, precision=prec, flags=tqc.FLAG_NO_RENORM)
    out = torch.empty(p.out_elems, dtype=torch.float64, device="cuda")
    p.contract(out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    entries, states = hss.product_states(net, [x.tolist() for x in sel])
    want = oracle.recon_states(net, states)
    scale = max(np.abs(want).max(), 1e-30)
    # FP32 (CUDA-core) and split-BF16 (tensor-core) arithmetic: relative errors
    # of a few 2^-24 and 2^-16 per product, amplified by cancellation
    assert np.abs(got[entries] - want).max() <= (1e-5 if prec == "fp32" else 1e-4) * scale + 1e-15
    pad = np.ones(got.size, bool)
    pad[entries] = False
    assert np.all(got[pad] == 0.0)
    p.close()
    sub.close()
    h.close()


@pytest.mark.parametrize("family", workloads.HSS_FAMILIES)
def test_p_hss_matches_oracle(family):
    net, _ = workloads.hss_circuit(family, 12)
    h = tqc.Network(net)
    sel, n_states = h.hss_select(32)
    sub = h.select(sel)
    p = tqc.Plan(sub, precision="auto", flags=tqc.FLAG_NO_RENORM)
    out = torch.empty(p.out_elems, dtype=torch.float64, device="cuda")
    p.contract(out)
    torch.cuda.synchronize()
    _, states = hss.product_states(net, [x.tolist() for x in sel])
    p_gpu = float(out.sum().item())
    p_or = float(oracle.recon_states(net, states).sum())
    print(f"{family}: |HSS| = {n_states}, P_HSS = {p_gpu:.6f} (oracle {p_or:.6f})")
    assert abs(p_gpu - p_or) <= 1e-5
    p.close()
    sub.close()
    h.close()
