"""Gate matrices in FP64, written from their definitions (Sec. 3.1, "Quantum Gates").

Two-qubit matrices act on the basis |a b> of their qubits (q0, q1) with row/column
index 2*a + b, i.e. q0 is the more significant factor (textbook form; for
controlled gates q0 is the control).  The paper prints the phase gate as
diag(1, e^{-j alpha}) (Sec. 4.2); we read it as the standard diag(1, e^{+i alpha})
(the sign is a convention; QFT followed by its inverse does not depend on it).
"""
import cmath
import math

import numpy as np

I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)
PAULI = {"I": I2, "X": X, "Y": Y, "Z": Z}

DIAGONAL = {"Z", "S", "SDG", "T", "TDG", "RZ", "P", "CZ", "CP"}


def rx(t):
    c, s = math.cos(t / 2), math.sin(t / 2)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def ry(t):
    c, s = math.cos(t / 2), math.sin(t / 2)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def rz(t):
    return np.array([[cmath.exp(-0.5j * t), 0], [0, cmath.exp(0.5j * t)]], dtype=np.complex128)


def phase(a):
    return np.array([[1, 0], [0, cmath.exp(1j * a)]], dtype=np.complex128)


def u3(t, p, l):
    """OpenQASM/Qiskit U(theta, phi, lambda)."""
    c, s = math.cos(t / 2), math.sin(t / 2)
    return np.array([[c, -cmath.exp(1j * l) * s],
                     [cmath.exp(1j * p) * s, cmath.exp(1j * (p + l)) * c]], dtype=np.complex128)


def controlled(u):
    m = np.eye(4, dtype=np.complex128)
    m[2:, 2:] = u
    return m


SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)


def matrix(kind, angles=()):
    """2x2 or 4x4 complex128 matrix of a gate."""
    if kind == "H":
        return H.copy()
    if kind == "X":
        return X.copy()
    if kind == "Y":
        return Y.copy()
    if kind == "Z":
        return Z.copy()
    if kind == "S":
        return phase(math.pi / 2)
    if kind == "SDG":
        return phase(-math.pi / 2)
    if kind == "T":
        return phase(math.pi / 4)
    if kind == "TDG":
        return phase(-math.pi / 4)
    if kind == "RX":
        return rx(angles[0])
    if kind == "RY":
        return ry(angles[0])
    if kind == "RZ":
        return rz(angles[0])
    if kind == "P":
        return phase(angles[0])
    if kind == "U3":
        return u3(*angles)
    if kind == "CX":
        return controlled(X)
    if kind == "CY":
        return controlled(Y)
    if kind == "CZ":
        return controlled(Z)
    if kind == "CP":
        return controlled(phase(angles[0]))
    if kind == "SWAP":
        return SWAP.copy()
    raise ValueError(kind)


def generator(kind):
    """G with dU/dtheta = -i/2 G U for the rotations exp(-i theta G / 2)."""
    return {"RX": X, "RY": Y, "RZ": Z}[kind]
