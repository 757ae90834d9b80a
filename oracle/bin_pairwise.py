"""Oracle C: a whole bin at once by FP64 pairwise contraction (numpy).

ORACLE: test infrastructure only.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s baseline legs may import it.  It shares no code with the
CUDA library and never imports it.

This is the tensor-network form of Eq. reconstruction (§III-B, Fig.
subcircuit_contraction) written the plain way: every subcircuit tensor keeps
one axis per cut (dimension 4) and one axis per output qubit (dimension 2).
Qubits outside the bin's free set are fixed by indexing their axis with the
fixed bit.  Two factors are then contracted at a time over all the cuts they
share (``numpy.tensordot``), always the pair whose result is smallest (pairs
that share a cut before pairs that do not; ties to the lowest pair of
positions), until one tensor over the free qubits is left.  The factor 1/2
per cut is applied once at the end.  Each qubit is an output of exactly one
subcircuit, so no qubit axis is ever summed: only the order of the sums in
the formula changes (distributivity).

It differs from oracle A (brute force per state) and oracle B (elimination
per state) in that the free qubits stay open, so a whole bin -- up to 2^28
entries -- is one computation.  It knows nothing of the library's layouts,
slicing or tiles.
"""
from __future__ import annotations

import numpy as np


def _restricted_factor(nd, free, fixed_bits):
    """(labels, tensor) of one node with its fixed output qubits indexed away.

    Labels: ('c', cut id) for a cut axis, ('q', qubit) for a free output."""
    t = nd.data.reshape((4,) * nd.n_cut + (2,) * nd.n_out)
    # bit k of x is out_qubits[k]; in C order the last axis is bit 0
    labels = [("c", int(c)) for c in nd.cut_ids] + [("q", int(nd.out_qubits[k])) for k in reversed(range(nd.n_out))]
    index, keep = [], []
    for lab in labels:
        if lab[0] == "q" and lab[1] not in free:
            index.append(int(fixed_bits[lab[1]]) if fixed_bits is not None else 0)
        else:
            index.append(slice(None))
            keep.append(lab)
    return keep, np.asarray(t[tuple(index)], dtype=np.float64)


def _dims(labels):
    return int(np.prod([4 if lab[0] == "c" else 2 for lab in labels], dtype=np.float64))


def recon_bin_pairwise(net, free_qubits=None, fixed_bits=None) -> np.ndarray:
    """P over the bin (2^F entries, FP64, entry bit i = i-th free qubit in
    ascending order; non-free qubit q carries fixed_bits[q], default 0)."""
    n = net.n_qubits
    free = sorted(range(n) if free_qubits is None else (int(q) for q in free_qubits))
    fset = set(free)
    factors = [_restricted_factor(nd, fset, fixed_bits) for nd in net.nodes]
    while len(factors) > 1:
        best = None
        for i in range(len(factors)):
            for j in range(i + 1, len(factors)):
                li, lj = set(factors[i][0]), set(factors[j][0])
                share = any(lab[0] == "c" for lab in li & lj)
                size = _dims(li ^ lj)
                key = (0 if share else 1, size, i, j)
                if best is None or key < best:
                    best = key
        _, _, i, j = best
        (la, ta), (lb, tb) = factors[i], factors[j]
        shared = [lab for lab in la if lab in lb]
        assert all(lab[0] == "c" for lab in shared), "a qubit axis appears in two factors"
        t = np.tensordot(ta, tb, axes=([la.index(x) for x in shared], [lb.index(x) for x in shared]))
        lab = [x for x in la if x not in shared] + [x for x in lb if x not in shared]
        factors = [f for k, f in enumerate(factors) if k not in (i, j)] + [(lab, t)]
    lab, t = factors[0]
    assert all(x[0] == "q" for x in lab), "every cut must appear in exactly two factors"
    # C order with the highest free qubit first: flat index bit i = free qubit i
    order = [lab.index(("q", q)) for q in reversed(free)]
    out = np.ascontiguousarray(np.transpose(t, order)).reshape(-1) if order else np.array(t, np.float64).reshape(1)
    out *= 2.0 ** -net.n_cuts          # exact: a power of two
    return out
