"""Arbitrary state lists (tqc_contract_states) against the FP64 oracles.

§VII-C reconstructs lists of arbitrary states.  Each state's probability is
checked element by element: oracle A (brute force over every cut
assignment) on the 30-qubit grid network and small networks, oracle B
(per-state elimination, spawned processes) on the 48-qubit QAOA bin network.

Gates: the fused form computes in FP32 on CUDA cores, so it meets the FP32
gate (1e-5 absolute per probability, and 1e-4 of the largest one).  The
per-state form runs the plan's own step kernels: the same FP32-class gate
when its tensor-core steps are split BF16, the 1e-3 total-variation gate
(over the listed states) when one is TF32."""
import numpy as np
import pytest

import oracle
from gen import Network, Node, tensors, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2502_03445_gb300 import tqc  # noqa: E402

FP32_ATOL = 1e-5
TC_TV = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def states_of(n_qubits, count, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, 1 << n_qubits, size=count, dtype=np.uint64)


def run_states(h, states, out_dtype=torch.float32, **kw):
    p = tqc.Plan(h, free_qubits=[], **kw)
    out = torch.full((len(states),), float("nan"), dtype=out_dtype, device="cuda")
    z = p.contract_states(states, out, want_z=True)
    torch.cuda.synchronize()
    d = p.describe()
    p.close()
    return out.cpu().numpy().astype(np.float64), z, d


def check_fp32(got, want):
    err = np.abs(got - want).max()
    assert err <= FP32_ATOL, err
    assert err <= 1e-4 * np.abs(want).max(), (err, np.abs(want).max())


def test_grid30_ten_thousand_states():
    """The 30-qubit grid network: 10^4 uniformly drawn states, fused form."""
    net = workloads.grid30(0)
    st = states_of(30, 10_000, 31)
    h = tqc.Network(net)
    got, z, d = run_states(h, st)
    assert d["states_form"] == "fused"
    z_or = oracle.total_mass(net)
    assert abs(z - z_or) <= 1e-9
    want = oracle.recon_states(net, st) / z_or
    check_fp32(got, want)
    # the same states through the full 2^30 bin
    p = tqc.Plan(h)
    full = torch.empty(p.out_elems, dtype=torch.float32, device="cuda")
    p.contract(full)
    fb = full[torch.from_numpy(st.astype(np.int64)).cuda()].double().cpu().numpy()
    assert np.abs(fb - got).max() <= 2 * FP32_ATOL
    p.close()
    h.close()


SMALL = [(13, 2, 4, 10), (14, 3, 5, 10), (15, 4, 7, 10), (16, 3, 8, 12), (14, 5, 8, 10), (16, 6, 9, 10)]


@pytest.mark.parametrize("seed", range(len(SMALL)))
def test_small_networks_fused(seed):
    """Shape-matched networks of 2-6 subcircuits (n, m, cuts, width as
    listed), with repeated states and FP64 output."""
    net = tensors.shape_matched_network(*SMALL[seed], seed=3700 + seed)
    st = states_of(net.n_qubits, 700, seed)
    st[::7] = st[0]                                  # duplicates
    h = tqc.Network(net)
    for out_dtype in (torch.float32, torch.float64):
        got, z, d = run_states(h, st, out_dtype)
        assert d["states_form"] == "fused"
        check_fp32(got, oracle.recon_states(net, st) / oracle.total_mass(net))
    h.close()


def test_zero_cuts_single_subcircuit_and_empty_list():
    rng = np.random.Generator(np.random.PCG64(8))
    a, b = rng.random(8), rng.random(16)
    outer = Network(7, 0, [Node([5, 0, 2], [], [], a / a.sum()), Node([1, 3, 6, 4], [], [], b / b.sum())])
    one = Network(5, 0, [Node([4, 0, 2, 1, 3], [], [], rng.random(32))])
    for net in (outer, one):
        net.check()
        st = states_of(net.n_qubits, 100, 9)
        h = tqc.Network(net)
        got, z, d = run_states(h, st)
        assert d["states_form"] == "fused"
        check_fp32(got, oracle.recon_states(net, st) / oracle.total_mass(net))
        p = tqc.Plan(h, free_qubits=[])
        p.contract_states(np.zeros(0, np.uint64), torch.empty(0, device="cuda"))
        p.close()
        h.close()


def test_no_renorm_and_uploads():
    """Raw probabilities with TQC_FLAG_NO_RENORM; new tensors are seen (the
    per-node tables are rebuilt when the tensors change)."""
    base = tensors.shape_matched_network(12, 3, 5, 9, seed=3800)
    nets = [tensors.random_data_network(base, s) for s in (1, 2)]
    st = states_of(12, 500, 3)
    h = tqc.Network(nets[0])
    p = tqc.Plan(h, free_qubits=[], flags=tqc.FLAG_NO_RENORM)
    out = torch.empty(len(st), dtype=torch.float64, device="cuda")
    for k, net in enumerate(nets):
        if k:
            for j, nd in enumerate(net.nodes):
                h.upload(j, nd.data)
        z = p.contract_states(st, out, want_z=True)
        torch.cuda.synchronize()
        want = oracle.recon_states(net, st)
        assert abs(z - oracle.total_mass(net)) <= 1e-9 * abs(oracle.total_mass(net))
        err = np.abs(out.cpu().numpy() - want).max()
        assert err <= 1e-4 * np.abs(want).max(), err
    p.close()
    h.close()


def test_qaoa48_per_state_form():
    """The 48-qubit QAOA bin network: single-state intermediates of 4^12
    floats run per state through the step kernels; 1024 uniformly drawn
    states against oracle B."""
    net = workloads.qaoa48(0)
    st = states_of(net.n_qubits, 1024, 48)
    h = tqc.Network(net)
    p = tqc.Plan(h, free_qubits=[])
    d = p.describe()
    assert d["states_form"] == "per-state"
    out = torch.empty(len(st), dtype=torch.float32, device="cuda")
    z = p.contract_states(st, out, want_z=True)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    want = oracle.recon_states_elim_pool(("gen.workloads", "qaoa48", (0,)), [int(s) for s in st]) / z
    assert abs(z - oracle.total_mass(net)) <= 1e-9 * abs(z)
    err = np.abs(got - want)
    tv = 0.5 * err.sum() / np.abs(want).sum()
    print(f"qaoa48 states: steps {[(s['log2_m'], s['log2_n'], s['log2_k'], s['class'], s['prec']) for s in d['steps']]}"
          f" max|err| {err.max():.3e} max|P| {np.abs(want).max():.3e} tv {tv:.3e}")
    assert err.max() <= FP32_ATOL
    if any(s["class"] == "tcgen05" and s["prec"] == "tf32" for s in d["steps"]):
        assert tv <= TC_TV
    else:
        # FP32-class steps summing up to 4^8 signed terms: within n_steps * 2^-12
        # of the mean absolute term mass per state (the reconstruction with
        # |T_j| in place of T_j, over 2^n), as for the full-size bins
        a = Network(net.n_qubits, net.n_cuts,
                    [Node(nd.out_qubits, nd.cut_ids, nd.cut_role, np.abs(nd.data)) for nd in net.nodes])
        scale = oracle.total_mass(a) / float(1 << net.n_qubits) / abs(z)
        assert err.max() <= max(1e-4 * np.abs(want).max(), len(d["steps"]) * 2.0 ** -12 * scale), (err.max(), scale)
    p.close()
    h.close()


def test_rejections():
    net = tensors.shape_matched_network(12, 3, 5, 9, seed=3900)
    h = tqc.Network(net)
    out = torch.empty(4, dtype=torch.float32, device="cuda")
    p = tqc.Plan(h)                                     # free qubits: not a single-state plan
    with pytest.raises(tqc.TqcError) as ei:
        p.contract_states([1, 2, 3, 4], out)
    assert ei.value.status == tqc.ERR_INVALID
    p.close()
    p = tqc.Plan(h, free_qubits=[], sliced=[1])
    with pytest.raises(tqc.TqcError) as ei:
        p.contract_states([1, 2, 3, 4], out)
    assert ei.value.status == tqc.ERR_UNSUPPORTED
    p.close()
    p = tqc.Plan(h, free_qubits=[])
    with pytest.raises(tqc.TqcError) as ei:
        p.contract_states([1, 2, 3, 1 << 12], out)      # a bit beyond n_qubits
    assert ei.value.status == tqc.ERR_INVALID
    p.close()
    h.close()
