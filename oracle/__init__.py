"""CPU FP64 oracle for the cut-network reconstruction.

ORACLE: test infrastructure only.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s ``cpu_baseline`` / ``--impl reference`` legs may import it.
It shares no code with the CUDA library and never imports it.

* **Oracle A** (:func:`recon_states`): the reconstruction formula (Eq.
  reconstruction, §II-A) with the factor 1/2 per cut, brute force over all
  4^|E| cut assignments per state, in plain C (``recon_bruteforce.c``).
* **Oracle B** (:func:`recon_states_elim`): per-state variable elimination
  in numpy FP64 -- fix x, each node becomes a tensor over its cuts, and the
  cuts are summed out one by one in ascending id.  A different algorithm from
  oracle A and from any contraction plan; used where 4^|E| per state is too
  slow, and checked against oracle A on small networks.
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


def _eliminate(factors, n_cuts: int) -> float:
    """Sum out cut variables 0..n_cuts-1 in order from a list of (axes, tensor)."""
    for c in range(n_cuts):
        bucket = [f for f in factors if c in f[0]]
        rest = [f for f in factors if c not in f[0]]
        union = sorted(set().union(*[set(ax) for ax, _ in bucket]))
        keep = [a for a in union if a != c]
        label = {a: i for i, a in enumerate(union)}
        ops = []
        for ax, t in bucket:
            ops += [t, [label[a] for a in ax]]
        ops.append([label[a] for a in keep])
        factors = rest + [(keep, np.einsum(*ops))]
    val = 1.0
    for ax, t in factors:
        assert not ax
        val *= float(t)
    return val


def recon_states_elim(net, states) -> np.ndarray:
    """Oracle B: per-state variable elimination in FP64."""
    out = np.empty(len(states), dtype=np.float64)
    for s_i, s in enumerate(states):
        factors = [(list(nd.cut_ids), _node_cut_tensor(nd, int(s))) for nd in net.nodes]
        out[s_i] = np.ldexp(_eliminate(factors, net.n_cuts), -net.n_cuts)
    return out


def total_mass(net) -> float:
    """Z = sum over all 2^n states of P(x), via per-node output sums."""
    factors = [(list(nd.cut_ids), nd.tensor().sum(axis=-1)) for nd in net.nodes]
    return float(np.ldexp(_eliminate(factors, net.n_cuts), -net.n_cuts))


def timed_sample(net, states, n_threads: int = 0):
    """(probabilities, seconds) of oracle A over ``states``."""
    t0 = time.perf_counter()
    p = recon_states(net, states, n_threads)
    return p, time.perf_counter() - t0
