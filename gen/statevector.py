"""Dense FP64 statevector simulation of small circuits (seeded input generation).

This module holds no reconstruction arithmetic.  It plays the part of the QPU
(the paper's subcircuit executions, §II-A) and of the "uncut circuit" that the
reconstruction must reproduce.  Conventions:

* qubit ``q`` is bit ``q`` of a basis-state index (little-endian);
* a gate is ``(kind, qubits, matrix)`` with ``matrix`` a 2x2 (one qubit) or
  4x4 (two qubits) complex unitary; for two-qubit gates the 4x4 matrix acts
  on the index ``b0 + 2*b1`` where ``b0`` is the bit of ``qubits[0]``.
"""
from __future__ import annotations

import numpy as np

SQ2 = np.sqrt(0.5)

I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
H = np.array([[1, 1], [1, -1]], dtype=np.complex128) * SQ2
PAULIS = (I2, X, Y, Z)          # basis order I, X, Y, Z (index 0..3)

# two-qubit gates, index b0 + 2*b1 (b0 = bit of qubits[0])
CZ = np.diag([1, 1, 1, -1]).astype(np.complex128)


def cnot() -> np.ndarray:
    """CNOT with control qubits[0], target qubits[1]."""
    m = np.zeros((4, 4), dtype=np.complex128)
    for b0 in range(2):
        for b1 in range(2):
            m[b0 + 2 * (b1 ^ b0), b0 + 2 * b1] = 1.0
    return m


def controlled(u: np.ndarray) -> np.ndarray:
    """Controlled-U, control qubits[0], target qubits[1]."""
    m = np.zeros((4, 4), dtype=np.complex128)
    m[0, 0] = 1.0
    m[2, 2] = 1.0            # control 0: target untouched (index 0 + 2*b1)
    for t_out in range(2):
        for t_in in range(2):
            m[1 + 2 * t_out, 1 + 2 * t_in] = u[t_out, t_in]
    return m


def rz(theta: float) -> np.ndarray:
    return np.diag([np.exp(-0.5j * theta), np.exp(0.5j * theta)])


def rx(theta: float) -> np.ndarray:
    c, s = np.cos(theta / 2), np.sin(theta / 2)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def ry(theta: float) -> np.ndarray:
    c, s = np.cos(theta / 2), np.sin(theta / 2)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def rzz(theta: float) -> np.ndarray:
    """exp(-i theta/2 Z(x)Z)."""
    ph = [np.exp(-0.5j * theta * (1 - 2 * (b0 ^ b1))) for b1 in range(2) for b0 in range(2)]
    return np.diag(ph).astype(np.complex128)


def haar_su2(rng: np.random.Generator) -> np.ndarray:
    """Haar-random SU(2) from a normalised 4-D Gaussian (a unit quaternion)."""
    q = rng.standard_normal(4)
    a, b, c, d = q / np.linalg.norm(q)
    return np.array([[a + 1j * b, c + 1j * d], [-c + 1j * d, a - 1j * b]], dtype=np.complex128)


def apply_1q(psi: np.ndarray, n: int, q: int, u: np.ndarray) -> np.ndarray:
    v = psi.reshape(1 << (n - q - 1), 2, 1 << q)
    return np.einsum("ab,ibj->iaj", u, v).reshape(-1)


def apply_2q(psi: np.ndarray, n: int, q0: int, q1: int, u: np.ndarray) -> np.ndarray:
    """Apply a 4x4 gate with index b0 + 2*b1 (b0 = bit q0, b1 = bit q1)."""
    t = psi.reshape((2,) * n)                 # axis k <-> qubit n-1-k
    a0, a1 = n - 1 - q0, n - 1 - q1
    u4 = u.reshape(2, 2, 2, 2)                # [b1_out, b0_out, b1_in, b0_in]
    t = np.moveaxis(t, (a1, a0), (0, 1))      # [b1, b0, rest...]
    t = np.tensordot(u4, t, axes=([2, 3], [0, 1]))
    t = np.moveaxis(t, (0, 1), (a1, a0))
    return t.reshape(-1)


def apply_gate(psi: np.ndarray, n: int, gate, qmap=None) -> np.ndarray:
    kind, qubits, mat = gate
    qs = [qmap[q] for q in qubits] if qmap is not None else list(qubits)
    if len(qs) == 1:
        return apply_1q(psi, n, qs[0], mat)
    return apply_2q(psi, n, qs[0], qs[1], mat)


def simulate(n: int, gates, psi0: np.ndarray | None = None) -> np.ndarray:
    """Statevector after applying ``gates`` to |0...0> (or ``psi0``)."""
    if psi0 is None:
        psi = np.zeros(1 << n, dtype=np.complex128)
        psi[0] = 1.0
    else:
        psi = np.array(psi0, dtype=np.complex128)
    for g in gates:
        psi = apply_gate(psi, n, g)
    return psi


def probabilities(n: int, gates) -> np.ndarray:
    psi = simulate(n, gates)
    return (psi.conj() * psi).real
