"""Subcircuit output tensors in the Pauli basis (input generation only).

Two builders, both seeded and both FP64:

``exact_network``
    Each subcircuit of a :class:`gen.cutter.CutCircuit` is simulated exactly.
    Its downstream cut qubits are prepared in the operators I, X, Y, Z (the
    linear combinations of the four physical initialisations |0>, |1>, |+>,
    |+i> that §II-A describes: I = r0 + r1, Z = r0 - r1, X = 2 r+ - r0 - r1,
    Y = 2 r+i - r0 - r1, which are exactly the Pauli matrices); its upstream
    cut qubits are measured in the Pauli observables I, X, Y, Z (outcome 0
    <-> eigenvalue +1); its remaining wires end as output bits ``x``:
    ``T[e][x] = Tr[(sigma_up(e) (x) |x><x|) U (sigma_down(e) (x) |0><0|) U^dag]``.

``pseudo_physical_tensor``
    For shapes too large to simulate, each physical variant (3 measurement
    bases per upstream cut, 4 initial states per downstream cut) gets a random
    exponential (Porter-Thomas-like) distribution over its measured bits; the
    same basis transforms as above then give the Pauli-basis tensor.  This
    keeps the trace identities, so the reconstructed distribution sums to 1.
"""
from __future__ import annotations

import numpy as np

from . import statevector as sv
from .cutter import CutCircuit
from .network import Network, Node

# stacked Pauli matrices S[e, row, col], e in I, X, Y, Z
_PAULI = np.stack(sv.PAULIS)

# upstream: measured-bit combination per basis index; variant basis 0 = Z, 1 = X, 2 = Y
# UP[e, basis, y]: coefficient of p_basis(y) in T^e
_UP = np.zeros((4, 3, 2))
_UP[0, 0] = [1, 1]           # I = p_Z(0) + p_Z(1)
_UP[1, 1] = [1, -1]          # X = p_X(0) - p_X(1)
_UP[2, 2] = [1, -1]          # Y = p_Y(0) - p_Y(1)
_UP[3, 0] = [1, -1]          # Z = p_Z(0) - p_Z(1)
# downstream: DOWN[e, init], init order |0>, |1>, |+>, |+i>
_DOWN = np.array([[1, 1, 0, 0],
                  [-1, -1, 2, 0],
                  [-1, -1, 0, 2],
                  [1, -1, 0, 0]], dtype=np.float64)


def subcircuit_tensor(sc):
    """Exact Pauli-basis tensor of one subcircuit.

    Returns ``(out_qubits, cut_ids, cut_role, data)`` with cut axes in
    ascending cut id and ``out_qubits`` ascending."""
    w = sc.width
    D = [i for i, s in enumerate(sc.segments) if s.init[0] == "cut"]
    U = [i for i, s in enumerate(sc.segments) if s.end[0] == "cut"]
    O = [i for i, s in enumerate(sc.segments) if s.end[0] == "out"]
    # statevectors psi_a = U |a on D, 0 elsewhere>
    nd = len(D)
    psis = []
    for a in range(1 << nd):
        idx = 0
        for t, q in enumerate(D):
            if (a >> t) & 1:
                idx |= 1 << q
        psi0 = np.zeros(1 << w, dtype=np.complex128)
        psi0[idx] = 1.0
        psis.append(sv.simulate(w, sc.gates, psi0))
    Psi = np.stack(psis).reshape((2,) * nd + (2,) * w)   # axes [a_{nd-1}..a_0][q_{w-1}..q_0]

    # integer labels for einsum
    lab = iter(range(100))
    a_ax = {t: next(lab) for t in range(nd)}
    b_ax = {t: next(lab) for t in range(nd)}
    q_ax = {q: next(lab) for q in range(w)}
    qp_ax = {q: (next(lab) if q in U else q_ax[q]) for q in range(w)}
    e_ax = {}
    for t, q in enumerate(D):
        e_ax[("d", t)] = next(lab)
    for q in U:
        e_ax[("u", q)] = next(lab)

    sub_psi = [a_ax[t] for t in reversed(range(nd))] + [q_ax[q] for q in reversed(range(w))]
    sub_psic = [b_ax[t] for t in reversed(range(nd))] + [qp_ax[q] for q in reversed(range(w))]
    ops = [Psi, sub_psi, Psi.conj(), sub_psic]
    for t in range(nd):            # sum_{a,b} sigma[a,b] <psi_b| . |psi_a>
        ops += [_PAULI, [e_ax[("d", t)], a_ax[t], b_ax[t]]]
    for q in U:                    # <psi_b| sigma_e |psi_a>: row index q', column q
        ops += [_PAULI, [e_ax[("u", q)], qp_ax[q], q_ax[q]]]

    # node axis order: cuts ascending by id, then output bits (MSB first in C order)
    cuts = []
    for t, q in enumerate(D):
        cuts.append((sc.segments[q].init[1], 1, e_ax[("d", t)]))
    for q in U:
        cuts.append((sc.segments[q].end[1], 0, e_ax[("u", q)]))
    cuts.sort()
    outs = sorted((sc.segments[q].end[1], q) for q in O)
    out_sub = [e for _, _, e in cuts] + [q_ax[q] for _, q in reversed(outs)]
    ops.append(out_sub)
    T = np.einsum(*ops, optimize="greedy")
    assert np.max(np.abs(T.imag), initial=0.0) < 1e-10
    return ([wq for wq, _ in outs], [c for c, _, _ in cuts], [r for _, r, _ in cuts],
            np.ascontiguousarray(T.real).reshape(-1))


def exact_network(cc: CutCircuit) -> Network:
    nodes = []
    for sc in cc.subs:
        oq, cid, role, data = subcircuit_tensor(sc)
        nodes.append(Node(oq, cid, role, data))
    net = Network(cc.n_qubits, cc.n_cuts, nodes, {"kind": "exact"})
    net.check()
    return net


def pseudo_physical_tensor(cut_role, n_out: int, rng: np.random.Generator, mass: float = 1.0) -> np.ndarray:
    """Random Pauli-basis tensor for a node with the given cut roles (in
    axis order) and ``n_out`` output bits.  Every physical variant's
    distribution over its measured bits has total ``mass`` (1 for a whole
    node; less when the node's tensor is restricted to one assignment of
    some output bits).  Returns float64 flat data."""
    ups = [i for i, r in enumerate(cut_role) if r == 0]
    downs = [i for i, r in enumerate(cut_role) if r == 1]
    u, d = len(ups), len(downs)
    # p[basis_0..basis_{u-1}, init_0..init_{d-1}, y_0..y_{u-1}, x]
    shape = (3,) * u + (4,) * d + (2,) * u + (1 << n_out,)
    p = rng.exponential(1.0, size=shape)
    p /= p.reshape((3 ** u) * (4 ** d), -1).sum(axis=1).reshape((3,) * u + (4,) * d + (1,) * (u + 1))
    p *= mass
    # upstream cuts contract (basis_t, y_t) -> e_t; downstream cuts contract init_t -> e_t
    labels = list(range(u)) + list(range(u, u + d)) + list(range(u + d, 2 * u + d)) + [2 * u + d]
    ops = [p, labels]
    eu = [2 * u + d + 1 + t for t in range(u)]
    ed = [3 * u + d + 1 + t for t in range(d)]
    for t in range(u):
        ops += [_UP, [eu[t], t, u + d + t]]
    for t in range(d):
        ops += [_DOWN, [ed[t], u + t]]
    # output axes in node order
    out = []
    ui = di = 0
    for r in cut_role:
        if r == 0:
            out.append(eu[ui]); ui += 1
        else:
            out.append(ed[di]); di += 1
    out.append(2 * u + d)
    ops.append(out)
    res = np.einsum(*ops, optimize="greedy")
    return np.ascontiguousarray(res, dtype=np.float64).reshape(-1)


def random_tree_edges(m: int, rng: np.random.Generator):
    order = rng.permutation(m)
    edges = []
    for k in range(1, m):
        edges.append((int(order[k]), int(order[rng.integers(0, k)])))
    return edges


def sample_shape(n_qubits: int, m: int, n_cuts: int, w_max: int, rng: np.random.Generator,
                 max_node_cuts: int | None = None, max_tries: int = 10000):
    """Shape-matched network skeleton: a random spanning tree plus extra
    random edges, directions from a random node order, initial qubits with sum n and widths
    w_j = i_j + d_j <= w_max.  Returns (edges[(up, down)], outs[j] list)."""
    if n_cuts < m - 1:
        raise ValueError("a connected network of m nodes needs at least m-1 cuts")
    for _ in range(max_tries):
        und = random_tree_edges(m, rng)
        while len(und) < n_cuts:
            a, b = rng.choice(m, size=2, replace=False)
            und.append((int(a), int(b)))
        # orient every cut from the earlier to the later node of a random
        # order: the cut graph is then a DAG, as time-ordered wire cuts are,
        # and the pseudo-physical trace identities make sum_x P(x) = 1 exact
        rank = rng.permutation(m)
        edges = [(a, b) if rank[a] < rank[b] else (b, a) for a, b in und]
        u = np.zeros(m, dtype=int)
        d = np.zeros(m, dtype=int)
        for a, b in edges:
            u[a] += 1
            d[b] += 1
        if max_node_cuts is not None and np.any(u + d > max_node_cuts):
            continue
        lo = np.maximum(0, u - d)
        hi = w_max - d
        if np.any(hi < lo) or lo.sum() > n_qubits or hi.sum() < n_qubits:
            continue
        i = lo.copy()
        rest = n_qubits - i.sum()
        while rest > 0:
            cand = np.nonzero(i < hi)[0]
            j = rng.choice(cand)
            i[j] += 1
            rest -= 1
        o = i + d - u
        perm = rng.permutation(n_qubits)
        outs, pos = [], 0
        for j in range(m):
            outs.append(sorted(int(q) for q in perm[pos:pos + o[j]]))
            pos += o[j]
        return edges, outs
    raise RuntimeError("sample_shape: no feasible network found")


def pseudo_physical_network(n_qubits: int, edges, outs, seed: int) -> Network:
    rng = np.random.Generator(np.random.PCG64(seed))
    m = len(outs)
    cuts = [[] for _ in range(m)]
    for cid, (a, b) in enumerate(edges):
        cuts[a].append((cid, 0))
        cuts[b].append((cid, 1))
    nodes = []
    for j in range(m):
        cl = sorted(cuts[j])
        role = [r for _, r in cl]
        data = pseudo_physical_tensor(role, len(outs[j]), rng)
        nodes.append(Node(list(outs[j]), [c for c, _ in cl], role, data))
    net = Network(n_qubits, len(edges), nodes, {"kind": "pseudo_physical", "seed": seed})
    net.check()
    return net


def bin_restricted_network(n_qubits: int, edges, outs, free_qubits, seed: int, meta=None) -> Network:
    """The network of one bin, drawn already restricted: node j keeps only
    its free output bits (the bin fixes the others), so its tensor has
    4^{c_j} * 2^{F_j} entries instead of 4^{c_j} * 2^{o_j} (§III-E-2 bins;
    full tensors at these widths would not fit in host memory).  Each
    physical variant is a random exponential distribution over its measured
    cut bits and free outputs with total mass 2^{-(fixed outputs of the
    node)}, the mean share of one fixed assignment.  Free qubits are
    renumbered 0..F-1 in ascending order; ``meta["free_qubits"]`` keeps the
    original ids."""
    free = sorted(int(q) for q in free_qubits)
    rank = {q: i for i, q in enumerate(free)}
    rng = np.random.Generator(np.random.PCG64(seed))
    m = len(outs)
    cuts = [[] for _ in range(m)]
    for cid, (a, b) in enumerate(edges):
        cuts[a].append((cid, 0))
        cuts[b].append((cid, 1))
    nodes = []
    for j in range(m):
        cl = sorted(cuts[j])
        role = [r for _, r in cl]
        f = [rank[q] for q in outs[j] if q in rank]
        n_fixed = len(outs[j]) - len(f)
        data = pseudo_physical_tensor(role, len(f), rng, mass=2.0 ** -n_fixed)
        nodes.append(Node(sorted(f), [c for c, _ in cl], role, data))
    net = Network(len(free), len(edges), nodes,
                  {"kind": "bin_restricted_pseudo_physical", "seed": seed, "free_qubits": free,
                   "n_qubits_full": n_qubits, **(meta or {})})
    net.check()
    return net


def restricted_shape_network(n_qubits: int, edges, outs, free_qubits, seed: int) -> Network:
    """The shape of ``bin_restricted_network`` with i.i.d. N(0,1) FP32-valued
    entries: fast to draw where only timing matters (planner training)."""
    free = sorted(int(q) for q in free_qubits)
    rank = {q: i for i, q in enumerate(free)}
    rng = np.random.Generator(np.random.PCG64(seed))
    m = len(outs)
    cuts = [[] for _ in range(m)]
    for cid, (a, b) in enumerate(edges):
        cuts[a].append((cid, 0))
        cuts[b].append((cid, 1))
    nodes = []
    for j in range(m):
        cl = sorted(cuts[j])
        f = sorted(rank[q] for q in outs[j] if q in rank)
        size = (4 ** len(cl)) << len(f)
        nodes.append(Node(f, [c for c, _ in cl], [r for _, r in cl],
                          rng.standard_normal(size, dtype=np.float32).astype(np.float64)))
    net = Network(len(free), len(edges), nodes, {"kind": "gaussian-restricted", "seed": seed, "free_qubits": free})
    net.check()
    return net


def shape_matched_network(n_qubits: int, m: int, n_cuts: int, w_max: int, seed: int,
                          max_node_cuts: int | None = None) -> Network:
    rng = np.random.Generator(np.random.PCG64(seed))
    edges, outs = sample_shape(n_qubits, m, n_cuts, w_max, rng, max_node_cuts)
    net = pseudo_physical_network(n_qubits, edges, outs, seed + 7919)
    net.meta.update({"edges": edges, "w_max": w_max})
    return net


def random_data_network(net: Network, seed: int) -> Network:
    """Same shape, i.i.d. N(0,1) entries (no physics; parity only)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nodes = [Node(nd.out_qubits, nd.cut_ids, nd.cut_role, rng.standard_normal(nd.data.size))
             for nd in net.nodes]
    return Network(net.n_qubits, net.n_cuts, nodes, {"kind": "gaussian", "seed": seed})


def random_shape_network(n_qubits: int, m: int, n_cuts: int, w_max: int, seed: int,
                         max_node_cuts: int | None = None) -> Network:
    """Shape-matched network with i.i.d. N(0,1) FP32-valued entries: fast to
    draw at sizes where only timing matters (cost-model training data)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    edges, outs = sample_shape(n_qubits, m, n_cuts, w_max, rng, max_node_cuts)
    cuts = [[] for _ in range(m)]
    for cid, (a, b) in enumerate(edges):
        cuts[a].append((cid, 0))
        cuts[b].append((cid, 1))
    nodes = []
    for j in range(m):
        cl = sorted(cuts[j])
        size = (4 ** len(cl)) << len(outs[j])
        nodes.append(Node(list(outs[j]), [c for c, _ in cl], [r for _, r in cl],
                          rng.standard_normal(size, dtype=np.float32).astype(np.float64)))
    net = Network(n_qubits, n_cuts, nodes, {"kind": "gaussian-shape", "seed": seed, "edges": edges})
    net.check()
    return net
