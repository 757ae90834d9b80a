"""Pins of the FP64 oracle against things other than itself.

* hand-derived golden fixtures (tests/golden);
* the brute-force statevector of the uncut circuit (|dP| <= 1e-12);
* closed forms: GHZ (1/2 at 0..0 and 1..1), W (1/n on weight-1 strings),
  an X gate through a cut identity wire, zero cuts (Kronecker product);
* sum_x P(x) = 1 for exact and pseudo-physical tensors;
* oracle B (variable elimination) against oracle A;
* every planted mistake in oracle A fails at least one pin.
"""
import json

import numpy as np
import pytest

import oracle
from gen import Network, Node, circuits, cutter, statevector as sv, tensors, workloads
from conftest import golden_path


def load_golden(name):
    with open(golden_path(name)) as f:
        g = json.load(f)
    nodes = [Node(nd["out_qubits"], nd["cut_ids"], nd["cut_role"], np.array(nd["data"], float))
             for nd in g["nodes"]]
    net = Network(g["n_qubits"], g["n_cuts"], nodes)
    net.check()
    return net, np.array(g["expected_P"])


@pytest.mark.parametrize("name", ["bell_one_cut.json", "x_identity_wire.json"])
def test_golden_fixtures(name):
    net, want = load_golden(name)
    np.testing.assert_allclose(oracle.recon_bin(net), want, atol=1e-15)
    states = list(range(1 << net.n_qubits))
    np.testing.assert_allclose(oracle.recon_states_elim(net, states), want, atol=1e-15)


def test_bell_fixture_matches_generated_tensors():
    """The cutter + exact builder reproduce the hand-derived Bell tensors."""
    n, gates = 2, [("h", (0,), sv.H), ("cx", (0, 1), sv.cnot())]
    cc = cutter.cut_circuit(n, gates, [0, 1])
    net = tensors.exact_network(cc)
    gold, _ = load_golden("bell_one_cut.json")
    for a, b in zip(net.nodes, gold.nodes):
        assert a.out_qubits == b.out_qubits and a.cut_ids == b.cut_ids and a.cut_role == b.cut_role
        np.testing.assert_allclose(a.data, b.data, atol=1e-15)


def test_line10_matches_statevector():
    net, (n, gates) = workloads.line10()
    P = oracle.recon_bin(net)
    np.testing.assert_allclose(P, sv.probabilities(n, gates), atol=1e-12, rtol=0)
    assert abs(P.sum() - 1) < 1e-12


@pytest.mark.parametrize("seed,n,depth,n_sub", [(1, 5, 3, 2), (2, 6, 4, 3), (3, 7, 3, 3),
                                                (4, 8, 3, 4), (5, 6, 2, 2), (6, 9, 3, 4)])
def test_random_circuits_match_statevector(seed, n, depth, n_sub):
    net, (nq, gates) = workloads.small_exact(seed, n=n, depth=depth, n_sub=n_sub, max_cuts=7)
    P = oracle.recon_bin(net)
    np.testing.assert_allclose(P, sv.probabilities(nq, gates), atol=1e-12, rtol=0)


def _cut(n, gates, groups):
    return tensors.exact_network(cutter.cut_circuit(n, gates, cutter.contiguous_partition(n, gates, groups)))


@pytest.mark.parametrize("n,groups", [(4, [[0, 1], [2, 3]]), (6, [[0, 1], [2, 3], [4, 5]]),
                                      (7, [[0, 1, 2], [3], [4, 5, 6]])])
def test_ghz_closed_form(n, groups):
    net = _cut(*circuits.ghz(n), groups)
    assert net.n_cuts >= 1
    P = oracle.recon_bin(net)
    want = np.zeros(1 << n)
    want[0] = want[-1] = 0.5
    np.testing.assert_allclose(P, want, atol=1e-13)


@pytest.mark.parametrize("n,groups", [(4, [[0, 1], [2, 3]]), (6, [[0, 1, 2], [3, 4, 5]]),
                                      (6, [[0, 1], [2, 3], [4, 5]])])
def test_w_closed_form(n, groups):
    net = _cut(*circuits.w_state(n), groups)
    assert net.n_cuts >= 1
    P = oracle.recon_bin(net)
    want = np.zeros(1 << n)
    for q in range(n):
        want[1 << q] = 1.0 / n
    np.testing.assert_allclose(P, want, atol=1e-13)


def test_identity_wire_cut():
    """A Haar gate, a cut, then an identity gate: P = |U|0>|^2."""
    rng = np.random.Generator(np.random.PCG64(11))
    u = sv.haar_su2(rng)
    gates = [("u", (0,), u), ("i", (0,), np.eye(2, dtype=complex))]
    cc = cutter.cut_circuit(1, gates, [0, 1])
    assert cc.n_cuts == 1
    P = oracle.recon_bin(tensors.exact_network(cc))
    np.testing.assert_allclose(P, np.abs(u[:, 0]) ** 2, atol=1e-15)


def test_zero_cuts_is_kronecker_of_marginals():
    rng = np.random.Generator(np.random.PCG64(2))
    a = rng.random(4)
    b = rng.random(8)
    net = Network(5, 0, [Node([0, 1], [], [], a), Node([2, 3, 4], [], [], b)])
    net.check()
    np.testing.assert_allclose(oracle.recon_bin(net), np.kron(b, a), rtol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_pseudo_physical_sums_to_one(seed):
    net = tensors.shape_matched_network(11, 3 + seed % 3, 3 + seed, 8, seed=100 + seed)
    P = oracle.recon_bin(net)
    assert abs(P.sum() - 1.0) < 1e-12
    assert abs(oracle.total_mass(net) - 1.0) < 1e-12


@pytest.mark.parametrize("seed", range(4))
def test_total_mass_equals_sum_over_states(seed):
    net = tensors.random_data_network(tensors.shape_matched_network(9, 3, 4, 7, seed=seed), seed)
    assert abs(oracle.total_mass(net) - oracle.recon_bin(net).sum()) < 1e-9


@pytest.mark.parametrize("seed", range(5))
def test_oracle_b_matches_oracle_a(seed):
    net = tensors.random_data_network(
        tensors.shape_matched_network(12, 3 + seed % 3, 4 + 2 * seed, 8, seed=200 + seed), seed)
    rng = np.random.Generator(np.random.PCG64(seed))
    states = [int(s) for s in rng.integers(0, 1 << 12, size=40)]
    a = oracle.recon_states(net, states)
    b = oracle.recon_states_elim(net, states)
    np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-12 * np.abs(a).max())


def test_bin_states_meaning():
    """A bin entry is the state whose free qubits carry the entry index."""
    net, (n, gates) = workloads.line10()
    full = sv.probabilities(n, gates)
    free = [1, 4, 6, 9]
    fixed = np.zeros(n, np.uint8)
    fixed[[0, 7]] = 1
    P = oracle.recon_bin(net, free, fixed)
    for i in range(16):
        s = (1 << 0) | (1 << 7)
        for b, q in enumerate(free):
            s |= ((i >> b) & 1) << q
        assert abs(P[i] - full[s]) < 1e-12


@pytest.mark.parametrize("mutation", [1, 2, 4, 8, 16])
def test_planted_mistakes_are_caught(mutation):
    """Each planted mistake in oracle A breaks a pin (statevector or golden)."""
    caught = False
    for net, (n, gates) in [workloads.line10(), workloads.small_exact(2, n=6, depth=4, n_sub=3)]:
        states = list(range(1 << n))
        P = oracle.recon_states(net, states, mutation=mutation)
        if np.abs(P - sv.probabilities(n, gates)).max() > 1e-9:
            caught = True
    for name in ["bell_one_cut.json", "x_identity_wire.json"]:
        g, want = load_golden(name)
        Pg = oracle.recon_states(g, list(range(1 << g.n_qubits)), mutation=mutation)
        if np.abs(Pg - want).max() > 1e-9:
            caught = True
    assert caught


# ---------------------------------------------------------------- oracle C (whole bin, pairwise FP64)
@pytest.mark.parametrize("name", ["bell_one_cut.json", "x_identity_wire.json"])
def test_oracle_c_golden_fixtures(name):
    net, want = load_golden(name)
    np.testing.assert_allclose(oracle.recon_bin_pairwise(net), want, atol=1e-15)


def test_oracle_c_matches_statevector_on_bins():
    """Full output and bins with fixed bits, against the uncut circuit's
    statevector (which shares nothing with either oracle)."""
    net, (n, gates) = workloads.line10()
    full = sv.probabilities(n, gates)
    np.testing.assert_allclose(oracle.recon_bin_pairwise(net), full, atol=1e-12, rtol=0)
    for free, ones in (([1, 4, 6, 9], [0, 7]), ([0, 2, 3, 5, 8], [9]), ([7], [1, 2, 3])):
        fixed = np.zeros(n, np.uint8)
        fixed[ones] = 1
        P = oracle.recon_bin_pairwise(net, free, fixed)
        idx = oracle.bin_states(n, free, fixed, np.arange(1 << len(free)))
        np.testing.assert_allclose(P, full[idx], atol=1e-12, rtol=0)


@pytest.mark.parametrize("n,groups", [(6, [[0, 1], [2, 3], [4, 5]]), (7, [[0, 1, 2], [3], [4, 5, 6]])])
def test_oracle_c_ghz_closed_form(n, groups):
    net = _cut(*circuits.ghz(n), groups)
    want = np.zeros(1 << n)
    want[0] = want[-1] = 0.5
    np.testing.assert_allclose(oracle.recon_bin_pairwise(net), want, atol=1e-13)


@pytest.mark.parametrize("seed", range(6))
def test_oracle_c_matches_oracle_a(seed):
    """Random-data networks (no physics), random bins: oracle C equals the
    brute-force formula entry by entry."""
    rng = np.random.Generator(np.random.PCG64(700 + seed))
    n = 11 + seed % 3
    net = tensors.random_data_network(
        tensors.shape_matched_network(n, 2 + seed % 4, 3 + seed % 4, 9, seed=700 + seed), seed)
    for F in (n, n - 3, 1, 0):
        free = sorted(rng.choice(n, size=F, replace=False).tolist())
        fixed = rng.integers(0, 2, size=n).astype(np.uint8)
        c = oracle.recon_bin_pairwise(net, free, fixed)
        a = oracle.recon_bin(net, free, fixed)
        assert c.shape == a.shape == (1 << F,)
        np.testing.assert_allclose(c, a, rtol=1e-11, atol=1e-13 * np.abs(a).max())


def test_oracle_c_zero_cuts_and_single_node():
    rng = np.random.Generator(np.random.PCG64(3))
    a, b = rng.random(4), rng.random(8)
    net = Network(5, 0, [Node([3, 1], [], [], a), Node([2, 0, 4], [], [], b)])
    net.check()
    np.testing.assert_allclose(oracle.recon_bin_pairwise(net), oracle.recon_bin(net), rtol=1e-15)
    one = Network(4, 0, [Node([2, 0, 3, 1], [], [], rng.random(16))])
    np.testing.assert_allclose(oracle.recon_bin_pairwise(one), oracle.recon_bin(one), rtol=1e-15)
