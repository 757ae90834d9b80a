"""Wire cutting by gate partition (input generation only).

The paper turns a circuit into a DAG of multi-qubit gates, attaches each
one-qubit gate to a neighbouring two-qubit gate and partitions the gates
(§VI-A-1).  Here the partition is given (or drawn by a simple contiguous
splitter); each wire is cut wherever two consecutive gates on it fall in
different subcircuits.  The upstream end of a cut is measured (in the
subcircuit holding the earlier gate), the downstream end is initialised (in
the subcircuit holding the later gate).

A subcircuit's local qubits are its wire *segments*: maximal runs of
consecutive gates on one wire inside that subcircuit.  Its width is the
number of segments.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Segment:
    wire: int
    init: tuple        # ("zero", None) or ("cut", cut_id)
    end: tuple         # ("out", wire) or ("cut", cut_id)


@dataclass
class Subcircuit:
    segments: list = field(default_factory=list)     # local qubit i = segments[i]
    gates: list = field(default_factory=list)        # (kind, local qubits, matrix)

    @property
    def width(self) -> int:
        return len(self.segments)


@dataclass
class CutCircuit:
    n_qubits: int
    subs: list
    n_cuts: int
    cut_ends: list     # cut id -> (upstream sub, downstream sub)


def attach_single_qubit_gates(n: int, gates, part2q: dict) -> list:
    """Complete a partition of the multi-qubit gates to all gates.

    A one-qubit gate joins the next multi-qubit gate on its wire, or the
    previous one if none follows; a wire with only one-qubit gates goes to
    subcircuit 0."""
    part = [None] * len(gates)
    for g, sub in part2q.items():
        part[g] = sub
    for q in range(n):
        idx = [g for g, (_, qs, _) in enumerate(gates) if q in qs]
        multi = [g for g in idx if len(gates[g][1]) > 1]
        for g in idx:
            if len(gates[g][1]) > 1:
                continue
            nxt = [h for h in multi if h > g]
            prv = [h for h in multi if h < g]
            if nxt:
                part[g] = part[nxt[0]]
            elif prv:
                part[g] = part[prv[-1]]
            else:
                part[g] = 0
    return part


def cut_circuit(n: int, gates, part) -> CutCircuit:
    """Cut the wires of ``(n, gates)`` along the gate partition ``part``."""
    m = max(part) + 1 if part else 1
    subs = [Subcircuit() for _ in range(m)]
    cut_ends = []
    cur = [None] * n                     # wire -> (sub, local qubit) of current segment
    for g, (kind, qs, mat) in enumerate(gates):
        s = part[g]
        local = []
        for q in qs:
            if cur[q] is None:           # first gate on the wire: circuit input
                subs[s].segments.append(Segment(q, ("zero", None), None))
                cur[q] = (s, subs[s].width - 1)
            elif cur[q][0] != s:         # the wire crosses subcircuits: a cut
                cid = len(cut_ends)
                ps, pl = cur[q]
                subs[ps].segments[pl].end = ("cut", cid)
                subs[s].segments.append(Segment(q, ("cut", cid), None))
                cur[q] = (s, subs[s].width - 1)
                cut_ends.append((ps, s))
            local.append(cur[q][1])
        subs[s].gates.append((kind, tuple(local), mat))
    for q in range(n):
        if cur[q] is None:               # an idle wire: its own segment in subcircuit 0
            subs[0].segments.append(Segment(q, ("zero", None), ("out", q)))
        else:
            s, l = cur[q]
            subs[s].segments[l].end = ("out", q)
    subs = [sc for sc in subs if sc.width > 0]
    if len(subs) != m:
        raise ValueError("empty subcircuit in partition")
    return CutCircuit(n, subs, len(cut_ends), cut_ends)


def contiguous_partition(n: int, gates, groups) -> list:
    """Partition by qubit groups: a multi-qubit gate goes to the group of its
    first qubit.  ``groups`` is a list of qubit lists."""
    owner = {}
    for gi, grp in enumerate(groups):
        for q in grp:
            owner[q] = gi
    part2q = {g: owner[qs[0]] for g, (_, qs, _) in enumerate(gates) if len(qs) > 1}
    return attach_single_qubit_gates(n, gates, part2q)


def widths(cc: CutCircuit):
    return [sc.width for sc in cc.subs]


def _partition_cost(n: int, wire_gates, lab, m: int, free):
    """(cuts, widths, node cut counts, node free outputs) of a labelling of
    the multi-qubit gates: a wire is cut wherever consecutive multi-qubit
    gates on it carry different labels (one cut end in each of the two
    subcircuits), every run of equal labels is one segment of that
    subcircuit, and a wire's output belongs to the label of its last gate."""
    cuts = 0
    w = np.zeros(m, dtype=np.int64)
    c = np.zeros(m, dtype=np.int64)
    f = np.zeros(m, dtype=np.int64)
    for q in range(n):
        seq = wire_gates[q]
        if not seq:
            w[0] += 1
            f[0] += q in free
            continue
        prev = lab[seq[0]]
        w[prev] += 1
        for g in seq[1:]:
            if lab[g] != prev:
                cuts += 1
                c[prev] += 1
                c[lab[g]] += 1
                w[lab[g]] += 1
                prev = lab[g]
        f[prev] += q in free
    return cuts, w, c, f


def anneal_partition(n: int, gates, m: int, w_max: int, seed: int, iters: int = 20000,
                     free_qubits=None, max_log2_elems: int | None = None) -> list:
    """A gate partition into ``m`` subcircuits of width <= ``w_max`` with few
    wire cuts, found by simulated annealing over the multi-qubit gates'
    labels.  Start: contiguous qubit blocks.  Energy: cuts, + 10 per qubit
    of excess width, + 100 per empty subcircuit, and, when
    ``max_log2_elems`` is given, + 10 per unit by which a node's
    bin-restricted tensor size log2(4^{c_j} 2^{F_j}) exceeds it (F_j = the
    node's outputs among ``free_qubits``).  This only generates inputs of the
    paper's cut sizes; it is not the paper's cut finder (§VI-A, Alg. 2/3).
    Returns the full per-gate partition (one-qubit gates attached)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    free = set(range(n) if free_qubits is None else free_qubits)
    multi = [g for g, (_, qs, _) in enumerate(gates) if len(qs) > 1]
    wire_gates = [[] for _ in range(n)]
    for g in multi:
        for q in gates[g][1]:
            wire_gates[q].append(g)
    lab = {g: min(gates[g][1][0] * m // n, m - 1) for g in multi}

    def penalty(cost):
        cuts, w, c, f = cost
        e = cuts + 10 * int(np.maximum(w - w_max, 0).sum()) + 100 * int((w == 0).sum())
        if max_log2_elems is not None:
            e += 10 * int(np.maximum(2 * c + f - max_log2_elems, 0).sum())
        return e

    e = penalty(_partition_cost(n, wire_gates, lab, m, free))
    best_e, best = e, dict(lab)
    for it in range(iters):
        temp = 2.0 * (1.0 - it / iters) + 0.05
        g = multi[int(rng.integers(len(multi)))]
        old, new = lab[g], int(rng.integers(m))
        if new == old:
            continue
        lab[g] = new
        e2 = penalty(_partition_cost(n, wire_gates, lab, m, free))
        if e2 <= e or rng.random() < np.exp((e - e2) / temp):
            e = e2
            if e < best_e:
                best_e, best = e, dict(lab)
        else:
            lab[g] = old
    cuts, w, c, f = _partition_cost(n, wire_gates, best, m, free)
    if np.any(w > w_max) or np.any(w == 0) or (
            max_log2_elems is not None and np.any(2 * c + f > max_log2_elems)):
        raise RuntimeError(f"anneal_partition: no feasible partition (widths {list(w)}, cuts {list(c)})")
    return attach_single_qubit_gates(n, gates, best)


def network_shape(cc: CutCircuit):
    """(edges, outs) of a cut circuit: ``edges[c] = (upstream sub, downstream
    sub)`` of cut c, ``outs[j]`` the sorted output wires of subcircuit j."""
    outs = [sorted(s.end[1] for s in sc.segments if s.end[0] == "out") for sc in cc.subs]
    return [tuple(e) for e in cc.cut_ends], outs
