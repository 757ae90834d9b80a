"""Pins of the cut-finder oracle (Alg. 2/3, Table I, Eq. qpu_runtime).

* the hand-derived run of tests/golden/cutfind_line3.json: the merging costs
  of the first iteration, the final partitions and the QPU runtimes;
* on seeded random circuits, the defining properties of the result: every
  subcircuit meets the hard limits (width, size), and no edge that joins two
  subcircuits can still merge within them and Q_max (the loop's stopping
  rule, checked by brute force over every edge);
* a planted mistake (widths counted per wire instead of per segment) breaks
  a pin."""
import json
import math

import numpy as np
import pytest

from conftest import golden_path
from oracle import cutfind as cf


def load():
    with open(golden_path("cutfind_line3.json")) as f:
        g = json.load(f)
    return g["n_qubits"], [tuple(x) for x in g["gates"]], g


def qmax(v):
    return math.inf if v == "inf" else float(v)


def test_graph_of_the_fixture():
    n, gates, g = load()
    _, edges, _ = cf.two_qubit_graph(n, gates)
    assert [list(e) for e in edges] == g["edges"]


@pytest.mark.parametrize("case", range(4))
def test_hand_derived_run(case):
    n, gates, g = load()
    c = g["cases"][case]
    multi, edges, wires = cf.two_qubit_graph(n, gates)
    if "first_iteration_q" in c:
        label = {x: x for x in multi}
        q = [cf.merging_cost(label, wires, a, b, c["w_max"], c["s_max"], c["k_t"]) for a, b in edges]
        np.testing.assert_allclose(q, c["first_iteration_q"], rtol=1e-12)
    lab = cf.greedy_graph_growing(n, gates, c["w_max"], c["s_max"], c["k_t"], qmax(c["q_max"]))
    part = cf.full_partition(n, gates, lab)
    assert part == c["partition"]
    subs, n_cuts = cf.subcircuits(n, gates, part)
    assert n_cuts == c["n_cuts"]
    if "subcircuits" in c:
        assert [list(s) for s in subs] == c["subcircuits"]
        assert abs(cf.qpu_runtime(subs) - c["t_qpu"]) <= 1e-12
        assert abs(cf.qpu_runtime(subs, n_qpus=10) - c["t_qpu"] / 10) <= 1e-12


def random_circuit(seed, n, n2q):
    rng = np.random.Generator(np.random.PCG64(seed))
    gates = []
    for _ in range(n2q):
        if rng.random() < 0.3:
            gates.append((int(rng.integers(n)),))
        a = int(rng.integers(n - 1))
        b = a + 1 if rng.random() < 0.7 else int(rng.integers(a + 1, n))
        gates.append((a, b))
    return gates


@pytest.mark.parametrize("seed,n,n2q,w_max,s_max,k_t,q_max",
                         [(1, 6, 14, 4, 6, 3, math.inf), (2, 8, 20, 5, 8, 4, 3.0), (3, 10, 30, 6, 12, 5, math.inf),
                          (4, 7, 18, 4, 5, 2, 2.5), (5, 9, 24, 5, 40, 6, math.inf)])
def test_result_properties(seed, n, n2q, w_max, s_max, k_t, q_max):
    gates = random_circuit(seed, n, n2q)
    lab = cf.greedy_graph_growing(n, gates, w_max, s_max, k_t, q_max)
    _, edges, wires = cf.two_qubit_graph(n, gates)
    width, size, _ = cf.partition_metrics(lab, wires)
    assert all(w <= w_max for w in width.values()) and all(s <= s_max for s in size.values())
    for a, b in edges:      # the loop stopped: no remaining edge is a valid merge
        if lab[a] != lab[b]:
            q = cf.merging_cost(lab, wires, a, b, w_max, s_max, k_t)
            assert not (q < math.inf and q <= q_max)
    part = cf.full_partition(n, gates, lab)
    subs, n_cuts = cf.subcircuits(n, gates, part)
    assert len(subs) == max(1, len(set(lab.values())))
    # cuts: every wire transition between subcircuits, each with one upstream and one downstream end
    assert sum(s[1] for s in subs) == sum(s[2] for s in subs) == n_cuts


def test_planted_width_mistake_is_caught(monkeypatch):
    """Counting one qubit per wire instead of per wire segment changes the
    hand-derived first-iteration costs."""
    n, gates, g = load()
    c = g["cases"][0]

    def per_wire(label, wires):
        width, size, cuts = orig(label, wires)
        for lab in width:
            width[lab] = sum(1 for seq in wires if any(label[x] == lab for x in seq))
        return width, size, cuts

    orig = cf.partition_metrics
    monkeypatch.setattr(cf, "partition_metrics", per_wire)
    multi, edges, wires = cf.two_qubit_graph(n, gates)
    label = {x: x for x in multi}
    q = [cf.merging_cost(label, wires, a, b, c["w_max"], c["s_max"], c["k_t"]) for a, b in edges]
    assert not np.allclose(q, c["first_iteration_q"])
