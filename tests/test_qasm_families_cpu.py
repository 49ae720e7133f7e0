"""The OpenQASM 2.0 front-end (sv_qasm_parse, Sec. 4.1's circuit input) and the
paper's other benchmark families (Sec. 5.1: AE, DJ, GHZ, Ising, QFT, QPE, SU2, VQC)
as seeded generators, on the CPU:

* QASM text written from every family parses back to the identical gate list;
* the parser's expressions, register layout, broadcast and the rzz / u2 rewrites are
  pinned (rzz against exp(-i t/2 Z x Z) from scipy, through the oracle's dense
  unitary);
* each family's defining property holds on the oracle (GHZ amplitudes, QPE and AE
  resolving an exact phase to its basis states, DJ's balanced oracle never returning
  |0...0>, a zero-time Ising evolution being the identity, unitarity);
* the C++ partitioner reproduces the oracle's partition of every family bit for bit,
  and partitions each family at 30-37 qubits (timed in bench.py against the paper's
  Python times).
"""
import math

import numpy as np
import pytest

import circuits as C
from oracle import dense as D
from oracle import partition as P
from oracle import statevector as S


@pytest.fixture(scope="module")
def sv():
    import __graft_entry__ as ge
    ge.build()
    import paper_2509_14098_gb300 as pkg
    return pkg


def _same_gates(a, b):
    assert a.n_qubits == b.n_qubits and len(a.gates) == len(b.gates)
    for x, y in zip(a.gates, b.gates):
        assert x.kind == y.kind and tuple(x.qubits) == tuple(y.qubits)
        assert tuple(x.angles) == tuple(y.angles)        # repr() round-trips doubles exactly


def _bind(c, params):
    """The circuit with its parameters substituted as fixed angles."""
    return C.Circuit(c.n_qubits, [C.Gate(g.kind, g.qubits, -1, c.angles_of(g, params)) for g in c.gates])


@pytest.mark.parametrize("name", sorted(C.FAMILIES))
def test_family_qasm_roundtrip(sv, name):
    c = C.FAMILIES[name](7)
    p = C.hea_params(c.n_params, 3) if c.n_params else None
    _same_gates(sv.parse_qasm(C.to_qasm(c, p)), _bind(c, p))


def test_qasm_roundtrip_other_workloads(sv):
    for c in (C.brickwork(6, 3, 2), C.random_circuit(5, 80, 7), C.qft_roundtrip(5)):
        _same_gates(sv.parse_qasm(C.to_qasm(c)), c)


def test_qasm_expressions_registers_broadcast(sv):
    text = """OPENQASM 2.0;
    include "qelib1.inc";   // ignored
    qreg a[2];
    qreg b[3];
    creg m[5];
    /* block
       comment */
    h b;
    rz(-pi/4 + 2*pi^2/3 - sqrt(2)*cos(0.5)) a[1];
    cx a[0], b[1];
    u2(0.25, -pi) a[0];
    u1(ln(2) / exp(1)) b[0];
    barrier a, b;
    measure a[0] -> m[0];
    cu1(-(1.5)) b[2], a[0];
    id a[1];
    swap a, b[0:1];
    """.replace("swap a, b[0:1];", "swap a[1], b[0];")
    c = sv.parse_qasm(text)
    assert c.n_qubits == 5
    want = [("H", (2,), ()), ("H", (3,), ()), ("H", (4,), ()),
            ("RZ", (1,), (-math.pi / 4 + 2 * math.pi ** 2 / 3 - math.sqrt(2) * math.cos(0.5),)),
            ("CX", (0, 3), ()), ("U3", (0,), (math.pi / 2, 0.25, -math.pi)),
            ("P", (2,), (math.log(2) / math.exp(1),)), ("CP", (4, 0), (-1.5,)), ("SWAP", (1, 2), ())]
    got = [(g.kind, g.qubits, g.angles) for g in c.gates]
    assert len(got) == len(want)
    for (k, q, a), (k2, q2, a2) in zip(got, want):
        assert k == k2 and q == q2 and np.allclose(a, a2, rtol=0, atol=1e-15)


def test_qasm_rzz_is_exp_zz(sv):
    scipy = pytest.importorskip("scipy.linalg")
    t = 0.8137
    c = sv.parse_qasm(f"qreg q[2]; rzz({t}) q[0],q[1];")
    assert [g.kind for g in c.gates] == ["CX", "RZ", "CX"]
    u = D.circuit_unitary(C.Circuit(2, [C.Gate(g.kind, g.qubits, -1, g.angles) for g in c.gates]))
    zz = np.diag([1.0, -1.0, -1.0, 1.0]).astype(complex)
    assert np.abs(u - scipy.expm(-0.5j * t * zz)).max() < 1e-14


@pytest.mark.parametrize("text,msg", [
    ("qreg q[2]; foo q[0];", "unsupported gate"),
    ("qreg q[2]; h q[2];", "out of range"),
    ("qreg q[2]; cx q[0];", "takes 2 qubits"),
    ("qreg q[2]; rz q[0];", "takes 1 parameters"),
    ("qreg q[2]; gate g a { h a; }", "not supported"),
    ("qreg q[2]; h r[0];", "unknown quantum register"),
    ("qreg q[2]; cx q[1],q[1];", "one qubit"),
    ("qreg q[2] h q[0];", "expected ';'"),
    ("creg c[2];", "no quantum register"),
    ("qreg q[2]; rz(1 +) q[0];", "expected an expression"),
])
def test_qasm_errors(sv, text, msg):
    with pytest.raises(sv.SvError) as e:
        sv.parse_qasm(text)
    assert msg in str(e.value)


def test_qasm_capacity(sv):
    import ctypes
    from paper_2509_14098_gb300 import _native as N
    src = b"qreg q[3]; h q;"
    nq, ng = ctypes.c_uint32(), ctypes.c_uint32()
    arr = (N.sv_gate * 2)()
    assert N.lib.sv_qasm_parse(src, arr, 2, ctypes.byref(nq), ctypes.byref(ng)) == N.SV_ERR_ARG
    assert nq.value == 3 and ng.value == 3


# ---------------------------------------------------------------------------
# the families' defining properties, on the oracle
# ---------------------------------------------------------------------------
def test_ghz_family():
    psi = S.simulate(C.FAMILIES["ghz"](6))
    assert abs(psi[0] - 2 ** -0.5) < 1e-15 and abs(psi[63] - 2 ** -0.5) < 1e-15


@pytest.mark.parametrize("seed", range(3))
def test_qpe_resolves_an_exact_phase(seed):
    n = 6
    c = C.qpe(n, seed, exact=True)
    psi = S.simulate(c)
    k = int(round(c.phase * (1 << (n - 1))))
    # counting register (qubits 0..n-2) holds k, the eigenvector qubit n-1 stays |1>
    assert abs(abs(psi[k | (1 << (n - 1))]) - 1.0) < 1e-12


def test_qpe_peaks_near_the_phase():
    n = 8
    c = C.qpe(n, 4)
    p = np.abs(S.simulate(c)) ** 2
    m = n - 1
    reg = p.reshape(2, 1 << m).sum(axis=0)
    best = int(np.argmax(reg))
    assert min(abs(best / (1 << m) - c.phase), 1 - abs(best / (1 << m) - c.phase)) <= 1.0 / (1 << m)
    assert reg[best] >= 4 / math.pi ** 2 - 1e-12      # QPE's guarantee for the nearest outcome


@pytest.mark.parametrize("seed", range(3))
def test_dj_balanced_never_returns_zero(seed):
    n = 7
    p = np.abs(S.simulate(C.dj(n, seed))) ** 2
    inputs_zero = p[0] + p[1 << (n - 1)]
    assert inputs_zero < 1e-24


def test_ising_zero_time_is_identity():
    c = C.ising(5, 3, dt=0.0)
    psi0 = C.random_state(5, 1)
    assert np.abs(S.simulate(c, None, psi0) - psi0).max() < 1e-14


def test_ae_resolves_an_exact_angle():
    n = 6
    m = n - 1
    j = 3
    p = math.sin(math.pi * j / (1 << m)) ** 2       # theta_p = 2 pi j / 2^m
    prob = np.abs(S.simulate(C.ae(n, p))) ** 2
    reg = prob.reshape(2, 1 << m).sum(axis=0)
    assert reg[j] + reg[(1 << m) - j] > 1 - 1e-12


@pytest.mark.parametrize("name", ["su2", "vqc", "ae", "ising"])
def test_families_preserve_norm(name):
    c = C.FAMILIES[name](6)
    p = C.hea_params(c.n_params, 2) if c.n_params else None
    assert abs(np.linalg.norm(S.simulate(c, p, C.random_state(6, 3))) - 1) < 1e-13


# ---------------------------------------------------------------------------
# partitioning the families
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", sorted(C.FAMILIES))
@pytest.mark.parametrize("L,nf", [(5, 0), (6, 4)])
def test_family_partitions_bit_exact(sv, name, L, nf):
    c = C.FAMILIES[name](10)
    stages, final = P.partition(c, L, range(min(nf, L)))
    assert P.validate(c, stages, L, range(min(nf, L)))[0]
    plan = sv.Plan(c, L, nf)
    order, fmap = plan.order()
    got, k = [], 0
    for mask, cnt in plan.stages():
        got.append((mask, order[k:k + cnt]))
        k += cnt
    assert got == [(sum(1 << b for b in loc), ids) for loc, ids in stages]
    assert fmap == final


@pytest.mark.parametrize("name", sorted(C.FAMILIES))
def test_family_partitions_at_paper_widths(sv, name):
    import time
    for n in (30, 37):
        c = C.FAMILIES[name](n)
        t0 = time.perf_counter()
        plan = sv.Plan(c, 11)
        dt = time.perf_counter() - t0
        assert len(plan.stages()) >= 1 and dt < 5.0
