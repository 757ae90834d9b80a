"""CPU FP64 oracle for the cut-network reconstruction.

ORACLE: test infrastructure only.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s ``cpu_baseline`` / ``--impl reference`` legs may import it.
It shares no code with the CUDA library and never imports it.

* **Oracle A** (:func:`recon_states`): the reconstruction formula (Eq.
  reconstruction, §II-A) with the factor 1/2 per cut, brute force over all
  4^|E| cut assignments per state, in plain C (``recon_bruteforce.c``).
* **Oracle B** (:func:`recon_states_elim`): per-state elimination in numpy
  FP64 -- fix x, each node becomes a tensor over its cuts, and factors are
  contracted two at a time over all the cuts they share (``tensordot``),
  always the pair with the smallest result first, until one scalar is left.
  Only the order of the sums in the formula changes (distributivity).  A
  different algorithm from oracle A, with no bit layouts, bins or tiles;
  used where 4^|E| per state is too slow, and checked against oracle A on
  small networks.
* :func:`total_mass`: Z = sum_x P(x) over the full output space.  Because the
  nodes' outputs partition the qubits, the sum over x splits into one sum per
  node, so Z = 2^{-|E|} sum_e prod_j S_j[e], S_j[e] = sum_x T_j[e][x].
* :func:`bin_states`: the meaning of an output vector for a bin -- entry i
  is the state whose free qubits (ascending) carry the bits of i and whose
  other qubits carry the fixed bits.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "recon_bruteforce.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle A with gcc (OpenMP).  Returns the library path."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.oracle_recon.restype = ctypes.c_int
        lib.oracle_recon.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
        lib.oracle_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def split_states(states):
    """Python ints (n <= 128 bits) -> (lo, hi) uint64 arrays."""
    st = [int(s) for s in states]
    lo = np.array([s & 0xFFFFFFFFFFFFFFFF for s in st], dtype=np.uint64)
    hi = np.array([s >> 64 for s in st], dtype=np.uint64)
    return lo, hi


def recon_states(net, states, n_threads: int = 0, mutation: int = 0) -> np.ndarray:
    """Oracle A: P(x) for each state x (python ints or a uint64 array)."""
    lib = _load()
    if isinstance(states, np.ndarray) and states.dtype == np.uint64:
        lo = np.ascontiguousarray(states)
        hi = np.zeros_like(lo)
    else:
        lo, hi = split_states(states)
    n_out = np.array([nd.n_out for nd in net.nodes], dtype=np.int32)
    n_cut = np.array([nd.n_cut for nd in net.nodes], dtype=np.int32)
    outq = np.array([q for nd in net.nodes for q in nd.out_qubits] or [0], dtype=np.int32)
    cids = np.array([c for nd in net.nodes for c in nd.cut_ids] or [0], dtype=np.int32)
    datas = [np.ascontiguousarray(nd.data, dtype=np.float64) for nd in net.nodes]
    ptrs = (ctypes.c_void_p * len(datas))(*[d.ctypes.data for d in datas])
    out = np.empty(len(lo), dtype=np.float64)
    rc = lib.oracle_recon(net.n_qubits, len(net.nodes), net.n_cuts,
                          n_out.ctypes.data, outq.ctypes.data, n_cut.ctypes.data, cids.ctypes.data,
                          ctypes.cast(ptrs, ctypes.c_void_p), len(lo), lo.ctypes.data, hi.ctypes.data,
                          out.ctypes.data, int(n_threads), int(mutation))
    if rc != 0:
        raise ValueError(f"oracle_recon failed ({rc})")
    return out


def bin_states(n_qubits: int, free_qubits, fixed_bits, idx) -> list:
    """States (python ints) of bin entries ``idx``.

    ``free_qubits`` ascending; ``fixed_bits[q]`` is the value of a non-free
    qubit q.  Bit i of the entry index is free qubit ``free_qubits[i]``."""
    free = list(free_qubits)
    base = 0
    fs = set(free)
    for q in range(n_qubits):
        if q not in fs and fixed_bits is not None and int(fixed_bits[q]):
            base |= 1 << q
    out = []
    for i in np.asarray(idx).reshape(-1).tolist():
        s = base
        for b, q in enumerate(free):
            if (i >> b) & 1:
                s |= 1 << q
        out.append(s)
    return out


def recon_bin(net, free_qubits=None, fixed_bits=None, n_threads: int = 0) -> np.ndarray:
    """Oracle A over a whole bin (default: every qubit free)."""
    if free_qubits is None:
        free_qubits = list(range(net.n_qubits))
    idx = np.arange(1 << len(free_qubits))
    return recon_states(net, bin_states(net.n_qubits, free_qubits, fixed_bits, idx), n_threads)


def _node_cut_tensor(nd, state: int) -> np.ndarray:
    x = 0
    for k, q in enumerate(nd.out_qubits):
        x |= ((state >> q) & 1) << k
    return nd.tensor()[..., x]


def _contract_pairs(factors) -> float:
    """Sum out every cut of a list of (axes, tensor) factors, in which each
    cut appears in exactly two factors: repeatedly contract the two factors
    whose result (the cuts in one but not both) is smallest -- ties to the
    lowest pair of positions -- over all the cuts they share."""
    factors = [(list(ax), np.asarray(t, dtype=np.float64)) for ax, t in factors]
    while len(factors) > 1:
        best = None
        for i in range(len(factors)):
            for j in range(i + 1, len(factors)):
                ai, aj = set(factors[i][0]), set(factors[j][0])
                if not ai & aj and best is not None:
                    continue
                size = len(ai ^ aj)
                if best is None or size < best[0] or (best[3] == 0 and ai & aj):
                    best = (size, i, j, len(ai & aj))
        _, i, j, _ = best
        (ax_i, t_i), (ax_j, t_j) = factors[i], factors[j]
        shared = [a for a in ax_i if a in ax_j]
        t = np.tensordot(t_i, t_j, axes=([ax_i.index(a) for a in shared], [ax_j.index(a) for a in shared]))
        ax = [a for a in ax_i if a not in shared] + [a for a in ax_j if a not in shared]
        factors = [f for k, f in enumerate(factors) if k not in (i, j)] + [(ax, t)]
    ax, t = factors[0]
    assert not ax, "every cut must appear in exactly two factors"
    return float(t)


def recon_states_elim(net, states) -> np.ndarray:
    """Oracle B: P(x) per state by pairwise elimination of the cut sums in FP64."""
    out = np.empty(len(states), dtype=np.float64)
    for s_i, s in enumerate(states):
        factors = [(list(nd.cut_ids), _node_cut_tensor(nd, int(s))) for nd in net.nodes]
        out[s_i] = np.ldexp(_contract_pairs(factors), -net.n_cuts)
    return out


def total_mass(net) -> float:
    """Z = sum over all 2^n states of P(x), via per-node output sums."""
    factors = [(list(nd.cut_ids), nd.tensor().sum(axis=-1)) for nd in net.nodes]
    return float(np.ldexp(_contract_pairs(factors), -net.n_cuts))


def timed_sample(net, states, n_threads: int = 0):
    """(probabilities, seconds) of oracle A over ``states``."""
    t0 = time.perf_counter()
    p = recon_states(net, states, n_threads)
    return p, time.perf_counter() - t0


from .bin_pairwise import recon_bin_pairwise  # noqa: E402,F401  (oracle C)
from .pool import recon_states_elim_pool  # noqa: E402,F401  (oracle B over spawned processes)
