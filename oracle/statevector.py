"""Gate-by-gate state-vector simulation in complex128 — the oracle for the hot path.

The exact result the partitioned method must reach is psi = U_G ... U_1 psi_0 with
the gates applied in the circuit's original flat order (Sec. 4.1: no permutation or
replacement of gates; Sec. 4.2: partitioning never breaks the sequential result).
Each gate is one tensor contraction over the dimensions of its qubits (Sec. 3.2,
the contraction xi = H . psi): the state is viewed as a rank-n tensor with one
size-2 axis per qubit and the gate's 2p-dimensional tensor is contracted into it.
Qubit q is bit q of the flat index, so it is tensor axis n-1-q in C order.
"""
import numpy as np

from . import gates as G


def _axis(n, q):
    return n - 1 - q


def apply_matrix(psi, n, qubits, u):
    """Contract a 2^p x 2^p gate matrix into the state over the given qubits.
    Row/column index of u: qubits[0] is the most significant bit."""
    p = len(qubits)
    t = psi.reshape([2] * n)
    ut = u.reshape([2] * (2 * p))                    # (out_0..out_{p-1}, in_0..in_{p-1})
    axes = [_axis(n, q) for q in qubits]
    r = np.tensordot(ut, t, axes=(list(range(p, 2 * p)), axes))   # out axes first, then the rest
    r = np.moveaxis(r, list(range(p)), axes)
    return np.ascontiguousarray(r).reshape(-1)


def apply_gate(psi, n, gate, angles):
    return apply_matrix(psi, n, gate.qubits, G.matrix(gate.kind, angles))


def simulate(circuit, params=None, psi0=None):
    """Apply every gate of the circuit in its original order to psi0 (default |0..0>)."""
    n = circuit.n_qubits
    if psi0 is None:
        psi = np.zeros(1 << n, dtype=np.complex128)
        psi[0] = 1.0
    else:
        psi = np.asarray(psi0, dtype=np.complex128).copy()
    for g in circuit.gates:
        psi = apply_gate(psi, n, g, circuit.angles_of(g, params))
    return psi


def simulate_prefix(circuit, k, params=None, psi0=None):
    """Apply only the first k gates (used for bounded CPU-baseline samples)."""
    n = circuit.n_qubits
    psi = np.asarray(psi0, dtype=np.complex128).copy()
    for g in circuit.gates[:k]:
        psi = apply_gate(psi, n, g, circuit.angles_of(g, params))
    return psi


def permute_qubits(psi, n, phys_of_wire):
    """Amplitude layout change: the returned vector holds, at index y, the amplitude of
    psi whose bit phys_of_wire[w] equals bit w of y (a pure bit permutation)."""
    idx = np.arange(1 << n, dtype=np.int64)
    src = np.zeros_like(idx)
    for w, p in enumerate(phys_of_wire):
        src |= ((idx >> w) & 1) << p
    return psi[src]


def dft_amplitude(psi, k, chunk=1 << 24):
    """One output amplitude of the QFT (little-endian, Sec. 5 QFT workload) from its
    definition y_k = 2^{-n/2} sum_x psi_x exp(2 pi i x k / 2^n), summed in chunks in
    FP64.  The exponent x*k is reduced mod 2^n in exact integer arithmetic."""
    N = len(psi)
    acc = 0j
    for s in range(0, N, chunk):
        x = np.arange(s, min(N, s + chunk), dtype=np.int64)
        ph = ((x * int(k)) % N).astype(np.float64) * (2.0 * np.pi / N)
        acc += np.sum(psi[s:s + len(x)].astype(np.complex128) * np.exp(1j * ph))
    return acc / np.sqrt(N)
