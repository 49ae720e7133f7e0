"""Pins for the oracle simulator against mathematics that does not use its code:
dense Kronecker unitaries, numpy's FFT, closed forms, invariants."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import circuits as C
from oracle import dense as D
from oracle import gates as GM
from oracle import statevector as S


@pytest.mark.parametrize("kind", C.KINDS)
def test_gate_unitary(kind):
    rng = np.random.default_rng(0)
    ang = tuple(rng.uniform(-3, 3, size=C.N_ANGLES.get(kind, 0)))
    u = GM.matrix(kind, ang)
    assert np.allclose(u @ u.conj().T, np.eye(u.shape[0]), atol=1e-14)


@pytest.mark.parametrize("t", [0.3, -1.7, 2.9])
def test_rotations_are_exponentials(t):
    # exp(-i t P / 2) computed by scipy, a different route from the closed forms
    for k, P in (("RX", GM.X), ("RY", GM.Y), ("RZ", GM.Z)):
        assert np.allclose(GM.matrix(k, (t,)), sla.expm(-0.5j * t * P), atol=1e-14)


def test_special_cases():
    t = 0.77
    assert np.allclose(GM.u3(t, -math.pi / 2, math.pi / 2), GM.rx(t))
    assert np.allclose(GM.u3(t, 0, 0), GM.ry(t))
    assert np.allclose(GM.u3(math.pi / 2, 0, math.pi), GM.H)
    assert np.allclose(GM.matrix("T") @ GM.matrix("T"), GM.matrix("S"))
    assert np.allclose(GM.matrix("S") @ GM.matrix("S"), GM.Z)
    assert np.allclose(GM.matrix("CP", (math.pi,)), GM.matrix("CZ"))
    assert np.allclose(GM.H @ GM.X @ GM.H, GM.Z)
    # RZ equals P up to a global phase
    assert np.allclose(GM.rz(t) * np.exp(0.5j * t), GM.phase(t))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_apply_matches_dense_kronecker(n):
    c = C.random_circuit(n, 40, seed=n)
    psi = C.random_state(n, 10 + n)
    ref = D.circuit_unitary(c) @ psi
    out = S.simulate(c, None, psi)
    assert np.abs(out - ref).max() < 1e-13


def test_dense_kronecker_paper_example():
    # Sec. 3.1: H on qubit 0 of three qubits.  With qubit q = index bit q the
    # Kronecker factor of qubit 0 is the rightmost one: I (x) I (x) H.
    u = D.embed(3, (0,), GM.H)
    assert np.allclose(u, np.kron(np.eye(4), GM.H))
    # controlled-X with control 0 and target 1 flips bit 1 where bit 0 is set
    u = D.embed(3, (0, 1), GM.matrix("CX"))
    for x in range(8):
        y = x ^ 2 if x & 1 else x
        assert u[y, x] == 1


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 10])
def test_qft_is_inverse_fft(n):
    psi = C.random_state(n, 3)
    out = S.simulate(C.qft(n), None, psi)
    assert np.abs(out - np.fft.ifft(psi, norm="ortho")).max() < 1e-13


def test_qft_basis_state_uniform_phases():
    n = 6
    psi = np.zeros(1 << n, dtype=complex)
    x = 13
    psi[x] = 1
    out = S.simulate(C.qft(n), None, psi)
    N = 1 << n
    assert np.allclose(np.abs(out), 1 / math.sqrt(N))
    k = np.arange(N)
    assert np.allclose(out, np.exp(2j * math.pi * x * k / N) / math.sqrt(N))


@pytest.mark.parametrize("n", [2, 3, 7])
def test_ghz(n):
    out = S.simulate(C.ghz(n))
    ref = np.zeros(1 << n, dtype=complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    assert np.abs(out - ref).max() < 1e-15


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_circuit_then_inverse_is_identity(seed):
    n = 5
    c = C.random_circuit(n, 60, seed)
    psi = C.random_state(n, seed)
    out = S.simulate(C.inverse(c), None, S.simulate(c, None, psi))
    assert np.abs(out - psi).max() < 1e-13
    out = S.simulate(C.qft_roundtrip(n), None, psi)
    assert np.abs(out - psi).max() < 1e-13


def test_norm_preserved():
    c, _, _ = C.workload("brick16")
    psi = S.simulate(c)
    assert abs(np.vdot(psi, psi).real - 1) < 1e-12


def test_permute_qubits_matches_swap_gates():
    n = 5
    psi = C.random_state(n, 4)
    # SWAP(0,3) then SWAP(1,4) as gates
    c = C.Circuit(n, [C.Gate("SWAP", (0, 3)), C.Gate("SWAP", (1, 4))])
    ref = S.simulate(c, None, psi)
    # the same result as a layout change: qubit w lives at phys[w]
    phys = [3, 4, 2, 0, 1]
    out = S.permute_qubits(psi, n, phys)
    assert np.allclose(out, ref)


def test_hea_counts():
    c = C.hea(28, 10)
    kinds = [g.kind for g in c.gates]
    assert (kinds.count("RY"), kinds.count("RZ"), kinds.count("CX"), c.n_params) == (280, 280, 270, 560)
    c = C.qft(30)
    kinds = [g.kind for g in c.gates]
    assert (kinds.count("H"), kinds.count("CP"), kinds.count("SWAP")) == (30, 435, 15)
    c = C.brickwork(32, 24, 3)
    kinds = [g.kind for g in c.gates]
    assert (kinds.count("U3"), kinds.count("CZ")) == (768, 372)


def test_dft_amplitude_definition():
    n = 9
    psi = C.random_state(n, 5)
    ref = np.fft.ifft(psi, norm="ortho")
    for k in (0, 1, 77, 511):
        assert abs(S.dft_amplitude(psi, k, chunk=100) - ref[k]) < 1e-13
