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
