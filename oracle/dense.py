"""Brute-force dense unitaries for small n (n <= 8), built from Kronecker products
the way Sec. 3.1 writes a gate on the full register (e.g. G_H = H (x) I (x) I).

Independent of statevector.py: every gate is embedded as a sum of Kronecker products
of 2x2 operators on each qubit, and the circuit unitary is the ordinary matrix
product of the embedded gates.  With qubit q = bit q of the index, the Kronecker
factor of qubit q sits at position n-1-q (highest qubit leftmost).
"""
import numpy as np

from . import gates as G


def _embed_ops(n, ops):
    """Kronecker product of per-qubit 2x2 operators (dict qubit -> matrix, identity elsewhere)."""
    m = np.ones((1, 1), dtype=np.complex128)
    for q in range(n - 1, -1, -1):
        m = np.kron(m, ops.get(q, G.I2))
    return m


def _unit(i, j):
    e = np.zeros((2, 2), dtype=np.complex128)
    e[i, j] = 1.0
    return e


def embed(n, qubits, u):
    """Full 2^n x 2^n matrix of a gate u on the given qubits."""
    if len(qubits) == 1:
        return _embed_ops(n, {qubits[0]: u})
    a, b = qubits
    full = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for ia in range(2):
        for ib in range(2):
            for ja in range(2):
                for jb in range(2):
                    c = u[2 * ia + ib, 2 * ja + jb]
                    if c != 0:
                        full += c * _embed_ops(n, {a: _unit(ia, ja), b: _unit(ib, jb)})
    return full


def circuit_unitary(circuit, params=None):
    n = circuit.n_qubits
    assert n <= 8, "dense brute force only for n <= 8"
    u = np.eye(1 << n, dtype=np.complex128)
    for g in circuit.gates:
        u = embed(n, g.qubits, G.matrix(g.kind, circuit.angles_of(g, params))) @ u
    return u
