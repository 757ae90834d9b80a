"""Cut finder oracle: Greedy Graph Growing (§VI-B, Alg. 2) with the edge
merging cost of Alg. 3 and Table I, and the QPU runtime of Eq. qpu_runtime.

ORACLE: test infrastructure only.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s baseline legs may import it.  It shares no code with the
library (whose C++ finder must produce the same partition) and never imports
it.

Readings of the paper taken here (it leaves these open):

* Graph (§VI-A-1).  Vertices are the two-qubit gates; an edge joins two of
  them when the later one is the next two-qubit gate on a wire of the
  earlier one (one edge per pair, ordered by (earlier, later) gate index).
  One-qubit gates take no part in the search.
* A partition's width w is its number of wire segments: on each wire, every
  maximal run of consecutive two-qubit gates inside the partition is one
  qubit of the subcircuit (a wire that leaves and comes back re-enters
  through a cut, on a new qubit).  Its size s is its number of two-qubit
  gates.  A cut is a wire between consecutive two-qubit gates in different
  partitions.
* Contraction edges of two neighbouring partitions P, N (they share a cut):
  K_{P,N} = |E_P u E_N|, the inner (shared) plus outer cuts of contracting
  them (§III-C).  K_trial of a trial merge T is the largest K_{T,N} over
  T's neighbours (0 without neighbours).
* Table I: a metric x with threshold T costs x / T when x <= T; above it a
  hard (quantum) metric -- width, size -- is not allowed, and the soft
  (classical) one -- contraction edges -- costs 4^{x-T} + 1.  Q_e is the sum
  of the three costs.
* Alg. 2 takes the valid edge of least Q_e with Q_e <= Q_max (ties: the
  lowest edge), merges its two partitions (the merged one keeps the lower
  label), recomputes the merging costs and repeats while a valid edge
  remains.
* One-qubit gates join the next two-qubit gate on their wire, else the
  previous one, else subcircuit 0 (§VI-A-1: they go with an adjacent
  two-qubit gate).  Subcircuits are numbered in order of their first gate.
* Eq. qpu_runtime with shots = 2^{w_i} limited to [2^10, 2^20] (§V: the
  shots equal the number of states of a subcircuit, within those limits),
  depth t_i = the number of layers of the subcircuit's gates (one- and
  two-qubit) scheduled as early as possible, divided by the number of QPUs
  that run subcircuits in parallel.
"""
from __future__ import annotations

import math


def two_qubit_graph(n, gates):
    """(two-qubit gate ids, edges as sorted (a, b) pairs, wire sequences)."""
    multi = [g for g, qs in enumerate(gates) if len(qs) == 2]
    wires = [[] for _ in range(n)]
    for g in multi:
        for q in gates[g]:
            wires[q].append(g)
    edges = set()
    for seq in wires:
        for a, b in zip(seq, seq[1:]):
            if a != b:
                edges.add((a, b))
    return multi, sorted(edges), wires


def partition_metrics(label, wires):
    """Per label: width (wire segments), size (gates), cut set."""
    width, size, cuts = {}, {}, {}
    for g, lab in label.items():
        size[lab] = size.get(lab, 0) + 1
        width.setdefault(lab, 0)
        cuts.setdefault(lab, set())
    cid = 0
    for q, seq in enumerate(wires):
        prev = None
        for g in seq:
            lab = label[g]
            if lab != prev:
                width[lab] += 1
                if prev is not None:
                    cuts[prev].add((q, cid))
                    cuts[lab].add((q, cid))
                    cid += 1
            prev = lab
    return width, size, cuts


def table_cost(x, t, hard):
    if x <= t:
        return x / t
    return math.inf if hard else 4.0 ** (x - t) + 1.0


def merging_cost(label, wires, a, b, w_max, s_max, k_t):
    """Q_e of merging the partitions of gates a and b (Alg. 3)."""
    la, lb = label[a], label[b]
    trial = {g: (la if lab == lb else lab) for g, lab in label.items()}
    width, size, cuts = partition_metrics(trial, wires)
    k_trial = 0
    for other, cs in cuts.items():
        if other != la and cs & cuts[la]:
            k_trial = max(k_trial, len(cuts[la] | cs))
    return (table_cost(width[la], w_max, True) + table_cost(size[la], s_max, True) +
            table_cost(k_trial, k_t, False))


def greedy_graph_growing(n, gates, w_max, s_max, k_t, q_max=math.inf):
    """Alg. 2: labels of the two-qubit gates (gate id -> partition label)."""
    multi, edges, wires = two_qubit_graph(n, gates)
    label = {g: g for g in multi}
    while True:
        best = None
        for a, b in edges:
            if label[a] == label[b]:
                continue
            q = merging_cost(label, wires, a, b, w_max, s_max, k_t)
            if q < math.inf and q <= q_max and (best is None or q < best[0]):
                best = (q, a, b)
        if best is None:
            return label
        _, a, b = best
        keep, gone = min(label[a], label[b]), max(label[a], label[b])
        for g in label:
            if label[g] == gone:
                label[g] = keep


def full_partition(n, gates, label):
    """Subcircuit of every gate, numbered in order of first gate."""
    part = [None] * len(gates)
    for g, lab in label.items():
        part[g] = lab
    per_wire = [[g for g, qs in enumerate(gates) if q in qs] for q in range(n)]
    for q in range(n):
        multi = [g for g in per_wire[q] if len(gates[g]) == 2]
        for g in per_wire[q]:
            if len(gates[g]) == 2:
                continue
            nxt = [h for h in multi if h > g]
            prv = [h for h in multi if h < g]
            part[g] = label[nxt[0]] if nxt else (label[prv[-1]] if prv else None)
    first = {}
    for g, lab in enumerate(part):
        if lab is not None and lab not in first:
            first[lab] = len(first)
    if not first:
        first[None] = 0
    return [first.get(lab, 0) for lab in part]


def subcircuits(n, gates, part):
    """Per subcircuit: (width, upstream cuts u, downstream cuts d, depth),
    and the cut count.  A wire is cut wherever consecutive gates on it sit
    in different subcircuits; a wire without gates is a qubit of
    subcircuit 0."""
    m = max(part) + 1 if part else 1
    width, up, down = [0] * m, [0] * m, [0] * m
    cur = [None] * n
    n_cuts = 0
    layer = [dict() for _ in range(m)]     # local depth per wire segment
    depth = [0] * m
    for g, qs in enumerate(gates):
        s = part[g]
        for q in qs:
            if cur[q] is None:
                width[s] += 1
            elif cur[q] != s:
                width[s] += 1
                up[cur[q]] += 1
                down[s] += 1
                n_cuts += 1
                layer[s][q] = 0        # a new local qubit, initialised by the cut
            cur[q] = s
        lvl = 1 + max(layer[s].get(q, 0) for q in qs)
        for q in qs:
            layer[s][q] = lvl
        depth[s] = max(depth[s], lvl)
    for q in range(n):
        if cur[q] is None:
            width[0] += 1
    return [(width[i], up[i], down[i], depth[i]) for i in range(m)], n_cuts


def qpu_runtime(subs, t_gate=1e-7, t_meas=1e-6, n_qpus=1, shots_log2=(10, 20)):
    """Eq. qpu_runtime: sum_i 3^{u_i} 4^{d_i} shots_i (t_i t_gate + t_meas) / n_qpus."""
    tot = 0.0
    for w, u, d, t in subs:
        shots = 2.0 ** min(max(w, shots_log2[0]), shots_log2[1])
        tot += 3.0 ** u * 4.0 ** d * shots * (t * t_gate + t_meas)
    return tot / n_qpus
