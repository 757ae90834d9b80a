"""Plain-data description of a cut network (shared input format).

A node is one subcircuit's output tensor in the Pauli basis (§II-A, §III-B):

* ``out_qubits[k]`` -- the original qubit that is bit ``k`` of the output
  index ``x`` (little-endian);
* ``cut_ids[i]`` -- the cut edge of tensor axis ``i`` (dimension 4, basis
  order I, X, Y, Z);
* ``cut_role[i]`` -- 0 if this node measures the cut (upstream end), 1 if it
  initialises it (downstream end);
* ``data`` -- float64, row-major ``[c_0][c_1]...[c_{n_cut-1}][x]``.

Every cut id in ``0..n_cuts-1`` appears in exactly two nodes, once in each
role, and the nodes' ``out_qubits`` partition ``0..n_qubits-1``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Node:
    out_qubits: list
    cut_ids: list
    cut_role: list
    data: np.ndarray

    @property
    def n_out(self) -> int:
        return len(self.out_qubits)

    @property
    def n_cut(self) -> int:
        return len(self.cut_ids)

    def tensor(self) -> np.ndarray:
        """``data`` viewed with one axis per cut and a final x axis."""
        return self.data.reshape((4,) * self.n_cut + (1 << self.n_out,))


@dataclass
class Network:
    n_qubits: int
    n_cuts: int
    nodes: list = field(default_factory=list)
    meta: dict = field(default_factory=dict)

    def check(self) -> None:
        seen = {}
        outs = []
        for j, nd in enumerate(self.nodes):
            assert nd.data.size == (4 ** nd.n_cut) << nd.n_out, "tensor size"
            for c, r in zip(nd.cut_ids, nd.cut_role):
                seen.setdefault(c, []).append((j, r))
            outs += list(nd.out_qubits)
        assert sorted(outs) == list(range(self.n_qubits)), "outputs must partition the qubits"
        assert sorted(seen) == list(range(self.n_cuts)), "cut ids must be 0..n_cuts-1"
        for c, ends in seen.items():
            assert len(ends) == 2 and sorted(r for _, r in ends) == [0, 1], f"cut {c} ends"
            assert ends[0][0] != ends[1][0], f"cut {c} joins a node to itself"

    def astype(self, dtype) -> "Network":
        nodes = [Node(nd.out_qubits, nd.cut_ids, nd.cut_role, nd.data.astype(dtype)) for nd in self.nodes]
        return Network(self.n_qubits, self.n_cuts, nodes, dict(self.meta))

    def shape_summary(self) -> list:
        return [(nd.n_cut, nd.n_out) for nd in self.nodes]
