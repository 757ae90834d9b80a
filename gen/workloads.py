"""Named synthetic workloads (seeded; seed = 1000 * workload + instance).

* ``line10``: 10-qubit line brickwork, depth 8, Haar SU(2) + CZ, cut into
  two 6-qubit subcircuits by 2 wire cuts; exact FP64 tensors.  Plain
  brickwork would cross the (4,5) boundary in four layers; the reading used
  here keeps that coupler in layer 4 only, so qubit 5's wire moves into the
  left subcircuit for that one gate and back (2 cuts, widths 6/6, 5 outputs
  each).
* ``grid30``: the shape of a 30-qubit (5x6) grid cut into 4 subcircuits of
  width 10 with 10 cuts -- a shape-matched network with pseudo-physical
  tensors (a real 5x6 depth-10 grid needs far more than 10 cuts at width 10).
* ``qaoa48``: 48-qubit QAOA p=1 on a seeded random 3-regular graph, cut by
  an annealed gate partition into 5 subcircuits of width <= 16 (16-24 wire
  cuts); one bin of 2^24 states (qubits 0-23 free, the rest fixed), node
  tensors drawn already restricted to the bin.
* ``grid64``: the shape of a 64-qubit (8x8) grid cut into 6 subcircuits of
  width <= 20 with 27 cuts; a stream of bins of 2^24 states (qubits 0-23
  free), each bin's node tensors drawn already restricted with its own seed.
* ``batch_recipe``: 256 independent networks of uneven sizes (n 16-28,
  2-8 subcircuits, 2-12 cuts) for the batched persistent launch.
* ``small_random``: tiny exact cut circuits for parity and oracle pins.
"""
from __future__ import annotations

import numpy as np

from . import circuits, cutter, statevector as sv, tensors
from .network import Network


def line_with_boundary(n: int, depth: int, seed: int, boundary: int, keep_layers):
    """Line brickwork whose coupler (boundary-1, boundary) is kept only in ``keep_layers``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gates = []
    for layer in range(depth):
        for q in range(n):
            gates.append(("u", (q,), sv.haar_su2(rng)))
        for q in range(layer % 2, n - 1, 2):
            if q == boundary - 1 and layer not in keep_layers:
                continue
            gates.append(("cz", (q, q + 1), sv.CZ))
    return n, gates


def line10(instance: int = 0):
    """Returns (network, (n, gates)) for the 10-qubit, 2-cut workload."""
    n, gates = line_with_boundary(10, 8, 1000 * 1 + instance, boundary=5, keep_layers=(4,))
    part = cutter.contiguous_partition(n, gates, [list(range(5)), list(range(5, 10))])
    cc = cutter.cut_circuit(n, gates, part)
    assert cc.n_cuts == 2 and cutter.widths(cc) == [6, 6], (cc.n_cuts, cutter.widths(cc))
    net = tensors.exact_network(cc)
    net.meta.update({"workload": "line10", "circuit": "line brickwork n=10 depth=8"})
    return net, (n, gates)


def grid30(instance: int = 0) -> Network:
    net = tensors.shape_matched_network(30, 4, 10, 10, seed=1000 * 2 + instance, max_node_cuts=7)
    net.meta.update({"workload": "grid30", "circuit": "shape of 5x6 grid, 4 subcircuits, width 10, 10 cuts"})
    return net


def qaoa48_shape(instance: int = 0):
    """(n, edges, outs) of the cut 48-qubit QAOA circuit ``instance``."""
    seed = 1000 * 4 + instance
    n, gates = circuits.qaoa_regular(48, seed)
    for m, tries in ((5, 0), (6, 0), (5, 1), (6, 1), (7, 0)):
        try:
            part = cutter.anneal_partition(n, gates, m, 16, seed=seed + 17 * m + 7919 * tries,
                                           free_qubits=range(24), max_log2_elems=24)
        except RuntimeError:
            continue
        cc = cutter.cut_circuit(n, gates, part)
        if 16 <= cc.n_cuts <= 24:
            edges, outs = cutter.network_shape(cc)
            return n, edges, outs
    raise RuntimeError(f"qaoa48 instance {instance}: no partition with 16..24 cuts")


def qaoa48(instance: int = 0, free_qubits=tuple(range(24))) -> Network:
    n, edges, outs = qaoa48_shape(instance)
    net = tensors.bin_restricted_network(n, edges, outs, free_qubits, seed=1000 * 4 + 500 + instance,
                                         meta={"workload": "qaoa48", "edges": edges,
                                               "circuit": "QAOA p=1, 3-regular graph, n=48"})
    return net


def qaoa48_timing(instance: int = 0, free_qubits=tuple(range(24))) -> Network:
    """The restricted shapes of ``qaoa48(instance)`` with Gaussian values
    (timing only: planner training and evaluation)."""
    n, edges, outs = qaoa48_shape(instance)
    net = tensors.restricted_shape_network(n, edges, outs, free_qubits, seed=1000 * 4 + 700 + instance)
    net.meta.update({"workload": "qaoa48-timing", "instance": instance, "edges": edges})
    return net


def grid64_shape(instance: int = 0):
    """(n, edges, outs) of the 64-qubit grid shape: 6 nodes, 27 cuts, width <= 20."""
    rng = np.random.Generator(np.random.PCG64(1000 * 5 + instance))
    for _ in range(1000):
        edges, outs = tensors.sample_shape(64, 6, 27, 20, rng, max_node_cuts=10)
        # keep every bin-restricted node tensor within 2^24 entries
        c = np.zeros(6, dtype=int)
        for a, b in edges:
            c[a] += 1
            c[b] += 1
        f = np.array([sum(q < 24 for q in o) for o in outs])
        if np.all(2 * c + f <= 24):
            return 64, edges, outs
    raise RuntimeError("grid64: no shape within the node size cap")


def grid64_bin(instance: int = 0, bin_index: int = 0, free_qubits=tuple(range(24))) -> Network:
    """Bin ``bin_index`` of the stream: same shape, own seeded tensors."""
    n, edges, outs = grid64_shape(instance)
    return tensors.bin_restricted_network(n, edges, outs, free_qubits,
                                          seed=1000 * 5 + 100 * (instance + 1) + bin_index,
                                          meta={"workload": "grid64", "bin": bin_index, "edges": edges,
                                                "circuit": "shape of 8x8 grid, 6 subcircuits, width <= 20, 27 cuts"})


def batch_recipe(count: int = 256, n_lo: int = 16, n_hi: int = 28, seed0: int = 3000,
                 max_node_elems: int = 1 << 24):
    """The batched workload: ``count`` independent networks with n ~ U{n_lo..n_hi},
    m ~ U{2..8}, |E| ~ U{max(2, m-1)..12}, widths up to n, i.i.d. Gaussian
    FP32-valued tensors.  Networks whose largest subcircuit tensor exceeds
    ``max_node_elems`` are redrawn.  Returns (networks, redraw count)."""
    rng = np.random.Generator(np.random.PCG64(seed0))
    nets, redraws = [], 0
    while len(nets) < count:
        n = int(rng.integers(n_lo, n_hi + 1))
        m = int(rng.integers(2, 9))
        cuts = int(rng.integers(max(2, m - 1), 13))
        seed = int(rng.integers(1 << 30))
        try:
            shape_rng = np.random.Generator(np.random.PCG64(seed))
            edges, outs = tensors.sample_shape(n, m, cuts, n, shape_rng, max_node_cuts=10)
        except RuntimeError:
            redraws += 1
            continue
        deg = [0] * m
        for a, b in edges:
            deg[a] += 1
            deg[b] += 1
        if max((4 ** deg[j]) << len(outs[j]) for j in range(m)) > max_node_elems:
            redraws += 1
            continue
        nets.append(tensors.random_shape_network(n, m, cuts, n, seed, max_node_cuts=10))
    return nets, redraws


# Two subcircuits of a 27-28-qubit network sharing one or two cut edges (a
# final step with K = 4 or 16): (n_qubits, cut edges, qubits of subcircuit 0
# as (kind, count), kind "lo" / "hi" = the lowest / highest qubits, "scr" = a
# seeded random draw; subcircuit 1 takes the rest).
SMALLK_CASES = {
    "16x12k4_rows_low": (28, [(0, 1)], ("lo", 16)),
    "16x12k4_cols_low": (28, [(0, 1)], ("hi", 16)),
    "16x12k4_scrambled": (28, [(0, 1)], ("scr", 16)),
    "23x4k16_cols_low": (27, [(0, 1)] * 2, ("hi", 23)),
    "16x12k16_rows_low": (28, [(0, 1)] * 2, ("lo", 16)),
    "16x12k16_scrambled": (28, [(0, 1)] * 2, ("scr", 16)),
}


def smallk_network(case: str, seed: int = 1) -> Network:
    """The network of one SMALLK_CASES entry, pseudo-physical tensors."""
    n, edges, (kind, cnt) = SMALLK_CASES[case]
    if kind == "lo":
        first = list(range(cnt))
    elif kind == "hi":
        first = list(range(n - cnt, n))
    else:
        first = sorted(int(q) for q in np.random.Generator(np.random.PCG64(7)).permutation(n)[:cnt])
    rest = [q for q in range(n) if q not in first]
    return tensors.pseudo_physical_network(n, edges, [first, rest], seed)


def planner_network(seed: int, kind: str = "g30"):
    """Timing-only networks for the learned planner (Gaussian FP32 values):
    ``g30`` -- 27-30 qubits, 4-6 subcircuits, m+5..m+7 cuts, widths <= 11
    (the 30-qubit grid workload's neighbourhood: sub-millisecond plans);
    ``m9`` -- 24-27 qubits, 9-12 subcircuits, m+2..m+4 cuts, widths <= 10
    (more subcircuits than TQC_PLANNER_AUTO plans exhaustively); ``small`` --
    20-24 qubits, 5-7 subcircuits, m+2..m+6 cuts, widths <= 12."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "g30":
        n, m = int(rng.integers(27, 31)), int(rng.integers(4, 7))
        cuts = int(rng.integers(m + 5, m + 8))
        return tensors.random_shape_network(n, m, cuts, 11, seed=seed, max_node_cuts=7)
    if kind == "m9":
        n, m = int(rng.integers(24, 28)), int(rng.integers(9, 13))
        cuts = int(rng.integers(m + 2, m + 5))
        return tensors.random_shape_network(n, m, cuts, 10, seed=seed, max_node_cuts=6)
    n, m = int(rng.integers(20, 25)), int(rng.integers(5, 8))
    cuts = int(rng.integers(m + 2, m + 7))
    return tensors.random_shape_network(n, m, cuts, 12, seed=seed, max_node_cuts=7)


HSS_FAMILIES = ("ghz", "w", "regular", "supremacy")


def hss_circuit(family: str, n: int = 20, m: int = 3, instance: int = 0):
    """The circuit families the paper evaluates heavy state selection on
    (§VII-B): GHZ, W, QAOA p=1 on a random 3-regular graph ("Regular") and a
    grid random circuit ("Supremacy", depth 5 on a rows x 5 grid), cut by the
    annealed gate partition into ``m`` subcircuits of width <= 13, with exact
    tensors.  Returns (network, (n, gates))."""
    seed = 1000 * 6 + 10 * HSS_FAMILIES.index(family) + instance
    if family == "ghz":
        n, gates = circuits.ghz(n)
    elif family == "w":
        n, gates = circuits.w_state(n)
    elif family == "regular":
        n, gates = circuits.qaoa_regular(n, seed)
    elif family == "supremacy":
        n, gates = circuits.grid(n // 5, 5, 5, seed)
    else:
        raise ValueError(family)
    part = cutter.anneal_partition(n, gates, m, 13, seed=seed + 5 + m, iters=4000)
    cc = cutter.cut_circuit(n, gates, part)
    net = tensors.exact_network(cc)
    net.meta.update({"workload": f"hss-{family}", "circuit": f"{family} n={n}, {m} subcircuits, {cc.n_cuts} cuts"})
    return net, (n, gates)


def random_cut_circuit(seed: int, n: int, depth: int, n_sub: int, family: str = "line"):
    """A small random circuit cut into ``n_sub`` contiguous qubit groups."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if family == "line":
        n, gates = circuits.line(n, depth, seed)
    else:
        raise ValueError(family)
    # random contiguous group boundaries
    cuts_at = sorted(rng.choice(np.arange(1, n), size=n_sub - 1, replace=False))
    bounds = [0] + list(cuts_at) + [n]
    groups = [list(range(bounds[i], bounds[i + 1])) for i in range(n_sub)]
    part = cutter.contiguous_partition(n, gates, groups)
    cc = cutter.cut_circuit(n, gates, part)
    return cc, (n, gates)


def small_exact(seed: int, n: int = 6, depth: int = 3, n_sub: int = 2, max_cuts: int = 8):
    """Exact network from a random line circuit; redraws until <= max_cuts cuts."""
    for k in range(100):
        cc, circ = random_cut_circuit(seed * 101 + k, n, depth, n_sub)
        if 0 < cc.n_cuts <= max_cuts:
            return tensors.exact_network(cc), circ
    raise RuntimeError("small_exact: no circuit within the cut limit")
