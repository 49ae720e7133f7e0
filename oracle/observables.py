"""Pauli-sum expectation values <psi|H|psi> with every Pauli factor applied explicitly."""
import numpy as np

from . import gates as G
from .statevector import apply_matrix


def apply_pauli_string(psi, n, s):
    out = psi
    for q, ch in enumerate(s):
        if ch != "I":
            out = apply_matrix(out, n, (q,), G.PAULI[ch])
    return out


def apply_observable(psi, obs):
    """lambda = H |psi> (the adjoint seed)."""
    lam = np.zeros_like(psi)
    for c, s in obs.terms:
        lam = lam + c * apply_pauli_string(psi, obs.n_qubits, s)
    return lam


def expval(psi, obs):
    return float(np.real(np.vdot(psi, apply_observable(psi, obs))))


def norm2(psi):
    return float(np.real(np.vdot(psi, psi)))
