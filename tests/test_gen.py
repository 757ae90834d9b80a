"""Pins of the input generators: simulator, cutter and tensor builders.

The simulator is pinned by textbook states and by an independent dense
Kronecker-product construction; the tensor builders by the trace identities
that the Pauli decomposition of a wire fixes (§II-A)."""
import itertools

import numpy as np
import pytest

from gen import circuits, cutter, statevector as sv, tensors, workloads


def dense_unitary(n, gates):
    """Full 2^n x 2^n matrix of a gate list, built from np.kron (independent
    of the reshaping simulator)."""
    U = np.eye(1 << n, dtype=np.complex128)
    for kind, qs, mat in gates:
        if len(qs) == 1:
            q = qs[0]
            full = np.kron(np.kron(np.eye(1 << (n - q - 1)), mat), np.eye(1 << q))
        else:
            q0, q1 = qs
            full = np.zeros((1 << n, 1 << n), dtype=np.complex128)
            for col in range(1 << n):
                b0, b1 = (col >> q0) & 1, (col >> q1) & 1
                for o0 in range(2):
                    for o1 in range(2):
                        row = col & ~(1 << q0) & ~(1 << q1) | (o0 << q0) | (o1 << q1)
                        full[row, col] += mat[o0 + 2 * o1, b0 + 2 * b1]
        U = full @ U
    return U


def test_bell_state():
    n, gates = 2, [("h", (0,), sv.H), ("cx", (0, 1), sv.cnot())]
    p = sv.probabilities(n, gates)
    np.testing.assert_allclose(p, [0.5, 0, 0, 0.5], atol=1e-15)


@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_ghz_state(n):
    p = sv.probabilities(*circuits.ghz(n))
    exp = np.zeros(1 << n)
    exp[0] = exp[-1] = 0.5
    np.testing.assert_allclose(p, exp, atol=1e-14)


@pytest.mark.parametrize("n", [2, 3, 4, 7])
def test_w_state(n):
    p = sv.probabilities(*circuits.w_state(n))
    exp = np.zeros(1 << n)
    for q in range(n):
        exp[1 << q] = 1.0 / n
    np.testing.assert_allclose(p, exp, atol=1e-14)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_simulator_matches_dense_kron(seed):
    n, gates = circuits.line(4, 3, seed)
    gates = gates + [("cx", (3, 0), sv.cnot()), ("rzz", (1, 3), sv.rzz(0.7))]
    psi = sv.simulate(n, gates)
    U = dense_unitary(n, gates)
    np.testing.assert_allclose(psi, U[:, 0], atol=1e-13)
    np.testing.assert_allclose(U.conj().T @ U, np.eye(1 << n), atol=1e-12)


def test_haar_su2_is_special_unitary():
    rng = np.random.Generator(np.random.PCG64(5))
    for _ in range(20):
        u = sv.haar_su2(rng)
        np.testing.assert_allclose(u.conj().T @ u, np.eye(2), atol=1e-14)
        assert abs(np.linalg.det(u) - 1) < 1e-13


def test_regular_graph_is_3_regular():
    rng = np.random.Generator(np.random.PCG64(3))
    edges = circuits.random_regular_graph(48, 3, rng)
    deg = np.zeros(48, int)
    for a, b in edges:
        assert a != b
        deg[a] += 1
        deg[b] += 1
    assert np.all(deg == 3) and len(set(edges)) == 72


def test_line10_cut_shape():
    net, _ = workloads.line10()
    assert net.n_cuts == 2
    assert [nd.n_out for nd in net.nodes] == [5, 5]
    assert [nd.n_cut for nd in net.nodes] == [2, 2]
    # qubit 5 leaves the right subcircuit and comes back: one cut each way
    roles = sorted(tuple(nd.cut_role) for nd in net.nodes)
    assert roles == [(0, 1), (1, 0)]


def test_cutter_counts_cuts_and_widths():
    n, gates = circuits.ghz(4)
    part = cutter.contiguous_partition(n, gates, [[0, 1], [2, 3]])
    cc = cutter.cut_circuit(n, gates, part)
    # cx(1,2) sits in group {0,1}: qubit 2 starts there, crosses to {2,3} for cx(2,3)
    assert cc.n_cuts == 1
    assert cutter.widths(cc) == [3, 2]


def _up_down(nd):
    return ([i for i, r in enumerate(nd.cut_role) if r == 0],
            [i for i, r in enumerate(nd.cut_role) if r == 1])


def check_trace_identities(net, physical=True):
    """sum_x T[e] with all upstream axes at I equals 2^d if every downstream
    axis is I and 0 otherwise (Tr of a Pauli is 0; Tr I = 2)."""
    for nd in net.nodes:
        S = nd.tensor().sum(axis=-1)
        ups, downs = _up_down(nd)
        for ed in itertools.product(range(4), repeat=len(downs)):
            idx = [0] * nd.n_cut
            for ax, v in zip(downs, ed):
                idx[ax] = v
            want = float(2 ** len(downs)) if all(v == 0 for v in ed) else 0.0
            assert abs(S[tuple(idx)] - want) < 1e-11, (tuple(idx), S[tuple(idx)], want)
        if physical and not downs:
            # measured-only node: |<sigma>| <= <I> per output state
            T = nd.tensor().reshape(4 ** nd.n_cut, -1)
            if nd.n_cut == 1:
                assert np.all(np.abs(T[1:]) <= T[0] + 1e-12)


@pytest.mark.parametrize("seed", range(6))
def test_exact_tensor_trace_identities(seed):
    net, _ = workloads.small_exact(seed, n=6, depth=3, n_sub=2 + seed % 2)
    check_trace_identities(net)


def test_line10_trace_identities():
    check_trace_identities(workloads.line10()[0])


@pytest.mark.parametrize("seed", range(4))
def test_pseudo_physical_trace_identities(seed):
    net = tensors.shape_matched_network(12, 3 + seed % 2, 4 + seed, 8, seed=seed)
    check_trace_identities(net, physical=False)


def test_shape_matched_widths():
    for seed in range(10):
        rng = np.random.Generator(np.random.PCG64(seed))
        edges, outs = tensors.sample_shape(30, 4, 10, 10, rng)
        u = np.zeros(4, int)
        d = np.zeros(4, int)
        for a, b in edges:
            u[a] += 1
            d[b] += 1
        o = np.array([len(x) for x in outs])
        w = o + u                 # width = outputs + measured cuts = initial + initialised
        assert np.all(w <= 10) and o.sum() == 30 and len(edges) == 10


def test_anneal_partition_matches_cut_circuit():
    n, gates = circuits.qaoa_regular(12, 77)
    part = cutter.anneal_partition(n, gates, 3, 8, seed=3, iters=3000)
    cc = cutter.cut_circuit(n, gates, part)
    assert len(cc.subs) == 3 and max(cutter.widths(cc)) <= 8
    # the annealer's own cut / width count agrees with the cutter
    multi = [g for g, (_, qs, _) in enumerate(gates) if len(qs) > 1]
    wire_gates = [[g for g in multi if q in gates[g][1]] for q in range(n)]
    cuts, w, c, f = cutter._partition_cost(n, wire_gates, {g: part[g] for g in multi}, 3, set(range(n)))
    assert cuts == cc.n_cuts and list(w) == cutter.widths(cc)
    edges, outs = cutter.network_shape(cc)
    assert sorted(q for o in outs for q in o) == list(range(n))
    assert list(c) == [sum(a == j for a, _ in edges) + sum(b == j for _, b in edges) for j in range(3)]
    assert list(f) == [len(o) for o in outs]


def _node_cuts(edges, m):
    c = np.zeros(m, dtype=int)
    for a, b in edges:
        c[a] += 1
        c[b] += 1
    return c


def test_qaoa48_shape_within_stated_sizes():
    n, edges, outs = workloads.qaoa48_shape(0)
    m = len(outs)
    assert n == 48 and 16 <= len(edges) <= 24 and m >= 5
    u = np.array([sum(a == j for a, _ in edges) for j in range(m)])
    o = np.array([len(x) for x in outs])
    assert np.all(o + u <= 16)                 # width = outputs + measured cuts
    assert sorted(q for x in outs for q in x) == list(range(48))
    f = np.array([sum(q < 24 for q in x) for x in outs])
    assert np.all(2 * _node_cuts(edges, m) + f <= 24)


def test_grid64_shape_within_stated_sizes():
    n, edges, outs = workloads.grid64_shape(0)
    m = len(outs)
    assert n == 64 and 24 <= len(edges) <= 30
    u = np.array([sum(a == j for a, _ in edges) for j in range(m)])
    o = np.array([len(x) for x in outs])
    assert np.all(o + u <= 20) and o.sum() == 64
    f = np.array([sum(q < 24 for q in x) for x in outs])
    assert np.all(2 * _node_cuts(edges, m) + f <= 24)


def test_bin_restricted_with_every_qubit_free_is_the_full_network():
    rng = np.random.Generator(np.random.PCG64(11))
    edges, outs = tensors.sample_shape(12, 3, 4, 8, rng)
    full = tensors.pseudo_physical_network(12, edges, outs, seed=5)
    restricted = tensors.bin_restricted_network(12, edges, outs, range(12), seed=5)
    for a, b in zip(full.nodes, restricted.nodes):
        assert a.out_qubits == b.out_qubits and a.cut_ids == b.cut_ids
        np.testing.assert_array_equal(a.data, b.data)


@pytest.mark.parametrize("seed", range(3))
def test_bin_restricted_trace_identities_scale_with_fixed_outputs(seed):
    """A node with k fixed outputs keeps the trace identities scaled by
    2^-k: each variant's distribution over the free outputs has mass 2^-k."""
    rng = np.random.Generator(np.random.PCG64(seed))
    edges, outs = tensors.sample_shape(14, 3, 5, 9, rng)
    free = sorted(rng.choice(14, size=8, replace=False).tolist())
    net = tensors.bin_restricted_network(14, edges, outs, free, seed=seed)
    assert net.n_qubits == 8 and net.meta["free_qubits"] == free
    for j, nd in enumerate(net.nodes):
        k = len(outs[j]) - nd.n_out
        S = nd.tensor().sum(axis=-1)
        ups, downs = _up_down(nd)
        for ed in itertools.product(range(4), repeat=len(downs)):
            idx = [0] * nd.n_cut
            for ax, v in zip(downs, ed):
                idx[ax] = v
            want = 2.0 ** (len(downs) - k) if all(v == 0 for v in ed) else 0.0
            assert abs(S[tuple(idx)] - want) < 1e-11
