"""Seeded circuit families shaped like the paper's benchmarks (§VII-B).

Every circuit is ``(n_qubits, gates)`` with gates as in :mod:`gen.statevector`.
Seeds follow numpy ``PCG64``.  The families:

* ``line``: Haar SU(2) on every qubit, then CZ on even pairs (even layers) or
  odd pairs (odd layers) -- the "Supremacy"-style brickwork on a line;
* ``grid``: the same on a rows x cols grid, the four coupler patterns
  (horizontal-even, horizontal-odd, vertical-even, vertical-odd) cycled;
* ``qaoa_regular``: QAOA p=1 on a random 3-regular graph (the "Regular"
  benchmark), angles U(0, pi);
* ``ghz`` and ``w_state``: the two closed-form benchmarks.
"""
from __future__ import annotations

import numpy as np

from . import statevector as sv


def line(n: int, depth: int, seed: int):
    rng = np.random.Generator(np.random.PCG64(seed))
    gates = []
    for layer in range(depth):
        for q in range(n):
            gates.append(("u", (q,), sv.haar_su2(rng)))
        start = layer % 2
        for q in range(start, n - 1, 2):
            gates.append(("cz", (q, q + 1), sv.CZ))
    return n, gates


def grid_couplers(rows: int, cols: int, pattern: int):
    """Pairs (q, q') of one coupler pattern; qubit id = r * cols + c."""
    pairs = []
    if pattern in (0, 1):              # horizontal, even / odd columns
        for r in range(rows):
            for c in range(pattern, cols - 1, 2):
                pairs.append((r * cols + c, r * cols + c + 1))
    else:                              # vertical, even / odd rows
        par = pattern - 2
        for r in range(par, rows - 1, 2):
            for c in range(cols):
                pairs.append((r * cols + c, (r + 1) * cols + c))
    return pairs


def grid(rows: int, cols: int, depth: int, seed: int):
    rng = np.random.Generator(np.random.PCG64(seed))
    n = rows * cols
    gates = []
    for layer in range(depth):
        for q in range(n):
            gates.append(("u", (q,), sv.haar_su2(rng)))
        for a, b in grid_couplers(rows, cols, layer % 4):
            gates.append(("cz", (a, b), sv.CZ))
    return n, gates


def random_regular_graph(n: int, degree: int, rng: np.random.Generator, max_tries: int = 1000):
    """Configuration model with rejection (no self loops, no multi-edges)."""
    if (n * degree) % 2:
        raise ValueError("n * degree must be even")
    for _ in range(max_tries):
        stubs = np.repeat(np.arange(n), degree)
        rng.shuffle(stubs)
        pairs = stubs.reshape(-1, 2)
        ok = all(a != b for a, b in pairs)
        edges = {tuple(sorted((int(a), int(b)))) for a, b in pairs}
        if ok and len(edges) == len(pairs):
            return sorted(edges)
    raise RuntimeError("random regular graph: rejection limit reached")


def qaoa_regular(n: int, seed: int, degree: int = 3):
    rng = np.random.Generator(np.random.PCG64(seed))
    edges = random_regular_graph(n, degree, rng)
    gamma, beta = rng.uniform(0.0, np.pi, size=2)
    gates = [("h", (q,), sv.H) for q in range(n)]
    for a, b in edges:
        gates.append(("rzz", (a, b), sv.rzz(gamma)))
    for q in range(n):
        gates.append(("rz", (q,), sv.rz(gamma)))
    for q in range(n):
        gates.append(("rx", (q,), sv.rx(2 * beta)))
    return n, gates


def ghz(n: int):
    gates = [("h", (0,), sv.H)]
    for q in range(n - 1):
        gates.append(("cx", (q, q + 1), sv.cnot()))
    return n, gates


def w_state(n: int):
    """|W_n> = (|10..0> + |010..0> + ... + |0..01>) / sqrt(n).

    X on qubit 0, then for i = 0..n-2 a controlled-RY moving all but a
    1/(n-i) share of the excitation forward, followed by a CNOT back."""
    gates = [("x", (0,), sv.X)]
    for i in range(n - 1):
        theta = 2.0 * np.arccos(np.sqrt(1.0 / (n - i)))
        gates.append(("cry", (i, i + 1), sv.controlled(sv.ry(theta))))
        gates.append(("cx", (i + 1, i), sv.cnot()))
    return n, gates
