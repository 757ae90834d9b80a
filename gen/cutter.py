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
