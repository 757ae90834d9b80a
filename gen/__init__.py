"""Seeded synthetic inputs for the cut-network reconstruction.

Shared by the oracle side (tests, CPU baseline) and the CUDA side (tests,
bench).  Holds circuit families, an FP64 statevector simulator standing in for
the QPUs, a gate-partition wire cutter, and the Pauli-basis tensor builders.
None of the reconstruction arithmetic lives here.
"""
from .network import Network, Node  # noqa: F401
from . import circuits, cutter, statevector, tensors, workloads  # noqa: F401
