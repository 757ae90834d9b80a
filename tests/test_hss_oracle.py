"""Pins of the heavy-state-selection oracle (§IV, §VII-A): hand-derived
selections, norm invariants, the selection's defining properties, the index
meaning of the selected network, and GHZ in closed form."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from gen import Network, Node, circuits, cutter, tensors, workloads
from oracle import hss

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hss_selection.json")


@pytest.mark.parametrize("case", json.load(open(GOLDEN))["cases"])
def test_selection_golden(case):
    sel = hss.select([np.array(v) for v in case["norms"]], case["s_max"])
    assert sel == case["expect"]
    assert math.prod(len(x) for x in sel) == case["n_states"]


def test_norm_invariants():
    net = tensors.shape_matched_network(12, 3, 5, 8, seed=31)
    norms = hss.state_norms(net)
    for nd, v in zip(net.nodes, norms):
        assert v.shape == (1 << nd.n_out,) and np.all(v >= 0)
        # the squares of the norms sum to the tensor's squared Frobenius norm
        assert abs((v ** 2).sum() - (nd.data ** 2).sum()) <= 1e-12 * (nd.data ** 2).sum()
    # a subcircuit without cuts: the norms are the absolute entries
    rng = np.random.Generator(np.random.PCG64(2))
    single = Network(3, 0, [Node([0, 1, 2], [], [], rng.standard_normal(8))])
    np.testing.assert_array_equal(hss.state_norms(single)[0], np.abs(single.nodes[0].data))


@pytest.mark.parametrize("seed", range(5))
def test_selection_properties(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    norms = [rng.random(1 << int(rng.integers(1, 6))) for _ in range(int(rng.integers(2, 5)))]
    total = math.prod(len(v) for v in norms)
    for s_max in (1, 2, 7, 40, total, total + 1):
        sel = hss.select(norms, s_max)
        prod = math.prod(len(x) for x in sel)
        assert prod >= min(s_max, total)
        # every subcircuit keeps its heaviest state
        assert all(int(np.argmax(v)) in x for v, x in zip(norms, sel))
        # beyond the seeds, the kept states are the heaviest of the pool
        kept = [v[i] for v, x in zip(norms, sel) for i in x if i != int(np.argmax(v))]
        dropped = [v[i] for v, x in zip(norms, sel) for i in range(len(v)) if i not in x]
        if kept and dropped:
            assert min(kept) >= max(dropped)
        # the last state added was needed: removing it leaves the product below s_max
        if prod > 1 and kept:
            lightest = min(kept)
            j = next(j for j, (v, x) in enumerate(zip(norms, sel)) for i in x
                     if i != int(np.argmax(v)) and v[i] == lightest)
            assert prod // len(sel[j]) * (len(sel[j]) - 1) < s_max


def test_product_state_indexing():
    # two subcircuits: A outputs qubits [0, 2], B outputs [1]; A keeps states 1, 2, 3, B keeps 1
    net = Network(3, 0, [Node([0, 2], [], [], np.zeros(4)), Node([1], [], [], np.zeros(2))])
    entries, states = hss.product_states(net, [[1, 2, 3], [1]])
    # A's index takes 2 bits (3 states, padded to 4), B's 0 bits
    assert entries == [0, 1, 2]
    # A state 1 -> qubit 0; state 2 -> qubit 2; state 3 -> qubits 0 and 2; B state 1 -> qubit 1
    assert states == [0b011, 0b110, 0b111]


def test_ghz_closed_form():
    """GHZ_8 cut into two halves: each half's heavy states are all-zeros and
    all-ones; keeping both per half reconstructs P_HSS = 1 with 4 of 256
    states (eta = 64), keeping one half's pair alone reconstructs 1/2."""
    n, gates = circuits.ghz(8)
    part = cutter.contiguous_partition(n, gates, [list(range(4)), list(range(4, 8))])
    net = tensors.exact_network(cutter.cut_circuit(n, gates, part))
    norms = hss.state_norms(net)
    sel = hss.select(norms, 4)
    for nd, x in zip(net.nodes, sel):
        assert x == [0, (1 << nd.n_out) - 1]
    _, states = hss.product_states(net, sel)
    p = oracle.recon_states(net, states)
    p_true = np.zeros(256)
    p_true[0] = p_true[255] = 0.5
    m = hss.metrics(p.sum(), len(states), 8, p_true)
    assert abs(m["P_HSS"] - 1) < 1e-12 and abs(m["r_P_HSS"] - 1) < 1e-12 and abs(m["eta_HSS"] - 64) < 1e-9
    sel2 = hss.select(norms, 2)
    _, states2 = hss.product_states(net, sel2)
    assert abs(oracle.recon_states(net, states2).sum() - 0.5) < 1e-12
