"""CPU FP64 oracle of heavy state selection (§IV, Alg. heavy_state_selection)
and of the metrics the paper evaluates it with (§VII-A: P_HSS, P_HSS^max,
Eq. hss_amplitude_ratio, r_|HSS|, Eq. hss_efficiency).

ORACLE: test infrastructure only (``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s baseline legs); it shares no code with the CUDA library.

* :func:`state_norms`: for every subcircuit and output state i, the L2 norm
  of its entries over all cut assignments, sqrt(sum_e T[e][i]^2).
* :func:`select`: the algorithm's steps in order -- seed each subcircuit
  with its heaviest state and take it out of the pool, sort the rest by norm
  (descending), then add states from the top while the product of the
  per-subcircuit counts is below s_max.  Ties (the paper is silent) go to the
  lower subcircuit, then the lower state index; the heaviest-state seed to
  the lowest index.
* :func:`product_states`: the meaning of an entry of the selected network's
  output: entry bits of subcircuit j (after those of subcircuits < j) index
  its ascending list of selected states; the full state is the OR of those
  states' output bits.
* :func:`metrics`: P_HSS, P_HSS^max, r_{P,HSS} = P_HSS / P_HSS^max,
  r_|HSS| = |HSS| / 2^n and eta_HSS = P_HSS / r_|HSS|.
"""
from __future__ import annotations

import math

import numpy as np


def state_norms(net):
    """List (one per subcircuit) of FP64 arrays of 2^{n_out} norms."""
    out = []
    for nd in net.nodes:
        t = nd.tensor().reshape(-1, 1 << nd.n_out).astype(np.float64)
        out.append(np.sqrt((t * t).sum(axis=0)))
    return out


def select(norms, s_max: int):
    """Heavy states per subcircuit (ascending lists) for the norms given."""
    chosen = [[] for _ in norms]
    pool = []
    for j, v in enumerate(norms):
        v = np.asarray(v, dtype=np.float64)
        best = int(np.argmax(v))            # first maximum: the lowest index
        chosen[j].append(best)
        pool += [(float(v[i]), j, i) for i in range(len(v)) if i != best]
    pool.sort(key=lambda c: (-c[0], c[1], c[2]))
    k = 0
    while math.prod(len(x) for x in chosen) < s_max and k < len(pool):
        _, j, i = pool[k]
        chosen[j].append(i)
        k += 1
    return [sorted(x) for x in chosen]


def index_bits(count: int) -> int:
    return 0 if count <= 1 else int(math.ceil(math.log2(count)))


def product_states(net, selection):
    """(entries, states): every valid entry of the selected network's output
    (python ints, ascending) and the full state it stands for."""
    kb = [index_bits(len(x)) for x in selection]
    if sum(kb) == 0:
        kb[0] = 1
    offs = np.cumsum([0] + kb[:-1]).tolist()
    entries, states = [0], [0]
    for j, (nd, sel) in enumerate(zip(net.nodes, selection)):
        # output bits of each selected state of subcircuit j, as full-state bits
        full = []
        for x in sel:
            s = 0
            for k, q in enumerate(nd.out_qubits):
                if (x >> k) & 1:
                    s |= 1 << q
            full.append(s)
        entries = [e | (r << offs[j]) for e in entries for r in range(len(sel))]
        states = [s | full[r] for s in states for r in range(len(sel))]
    order = np.argsort(entries, kind="stable")
    return [entries[i] for i in order], [states[i] for i in order]


def metrics(p_hss: float, n_states: int, n_qubits: int, p_true):
    """The paper's HSS metrics; p_true: the error-free distribution (any order)."""
    top = np.sort(np.asarray(p_true, dtype=np.float64))[::-1][:n_states]
    p_max = float(top.sum())
    r_size = n_states / float(2 ** n_qubits)
    return {"P_HSS": float(p_hss), "P_HSS_max": p_max, "r_P_HSS": float(p_hss) / p_max if p_max > 0 else 0.0,
            "r_size": r_size, "eta_HSS": float(p_hss) / r_size, "n_states": int(n_states)}
