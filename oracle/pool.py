"""Oracle B over many states in parallel host processes.

ORACLE: test infrastructure only.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s baseline legs may import it.

Each worker is a *spawned* process (never forked: a fork of a process that
has touched the GPU can hang) with single-threaded BLAS.  It rebuilds the
network from a seeded generator spec ``(module, function, args)`` -- e.g.
``("gen.workloads", "qaoa48", (0,))`` -- instead of receiving the tensors
through a pipe, then evaluates its share of the states with
:func:`oracle.recon_states_elim`.  The arithmetic is oracle B's, unchanged.
"""
from __future__ import annotations

import importlib
import multiprocessing as mp
import os

import numpy as np

_NET = None


def _init(spec):
    global _NET
    mod, fn, args = spec
    _NET = getattr(importlib.import_module(mod), fn)(*args)


def _work(states):
    from . import recon_states_elim
    return recon_states_elim(_NET, states)


def recon_states_elim_pool(spec, states, procs: int = 0) -> np.ndarray:
    """Oracle B for ``states`` (python ints) of the network ``spec`` builds."""
    states = [int(s) for s in states]
    if not states:
        return np.zeros(0)
    procs = procs or min(len(states), os.cpu_count() or 1, 32)
    chunks = [states[i::procs] for i in range(procs)]
    keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in keep:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(procs, initializer=_init, initargs=(spec,)) as pool:
            parts = pool.map(_work, chunks)
    finally:
        for k, v in keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    out = np.empty(len(states))
    for i, p in enumerate(parts):
        out[i::procs] = p
    return out
