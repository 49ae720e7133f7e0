"""The host planner's output executed on the CPU (no GPU): `tests/host_emu/stage_emu.cpp`
runs the library's SWAP relabel, closeness-centrality partition, lowering (register
groups, micro-ops, diagonal sinking, twiddles, phase slots, pair phases folded into
real butterflies; adjoint programs with their gradient ops) and packing, then executes
the packed programs in double precision, tile by tile and thread by thread.  The
forward state must match the CPU oracle's gate-by-gate result, and the adjoint
program's E and gradient the oracle's expectation value and parameter-shift gradient:
within 1e-10 for the complex128 packing (FP64 matrices and angles), within the
complex64 tolerances for the complex64 packing (FP32 matrices, 32-bit fixed-point
phase turns)."""
import os
import struct
import subprocess

import numpy as np
import pytest

import circuits as C
from oracle import gradients as GR
from oracle import observables as O
from oracle import statevector as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2509_14098_gb300", "csrc")


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    import __graft_entry__ as ge
    ge.build()
    from paper_2509_14098_gb300 import _native as N
    global GATE_CODES
    GATE_CODES = N.GATE_CODES                       # the C ABI's gate kind codes
    exe = str(tmp_path_factory.mktemp("emu") / "stage_emu")
    cmd = ["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "host_emu", "stage_emu.cpp"),
           os.path.join(CSRC, "partition.cpp"), os.path.join(CSRC, "lower.cpp"),
           os.path.join(CSRC, "gemm_plan.cpp"), os.path.join(CSRC, "hier_plan.cpp"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True)
    return exe


def run_emu(exe, tmp_path, circ, L, n_fixed, params, psi0, elem_bytes, rmax=4, obs=None, bind=False, gemm=False,
            fuse=False, hier=False):
    n = circ.n_qubits
    params = [] if params is None else list(params)
    buf = [struct.pack("<7i", n, L, n_fixed, len(params), len(circ.gates), elem_bytes, rmax)]
    buf.append(struct.pack(f"<{len(params)}d", *params))
    for g in circ.gates:
        q = list(g.qubits) + [-1] * (2 - len(g.qubits))
        a = list(g.angles) + [0.0] * (3 - len(g.angles))
        buf.append(struct.pack("<5i3d", GATE_CODES[g.kind], len(g.qubits), q[0], q[1], g.param, *a))
    buf.append(np.ascontiguousarray(psi0, dtype=np.complex128).tobytes())
    if obs is not None:
        buf.append(struct.pack("<i", len(obs.terms)))
        for c, ps in obs.terms:
            buf.append(struct.pack("<d", c) + bytes("IXYZ".index(ch) for ch in ps))
    fin, fout = tmp_path / "in.bin", tmp_path / "out.bin"
    fin.write_bytes(b"".join(buf))
    mode = "hier" if hier else ("gemm" if gemm else ("bind" if bind else ("grad" if obs is not None else ("fuse" if fuse else "fwd"))))
    r = subprocess.run([exe, mode, str(fin), str(fout)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    raw = fout.read_bytes()
    if gemm or hier:
        return int(np.frombuffer(raw[:8], dtype=np.float64)[0]), np.frombuffer(raw[8:], dtype=np.complex128)
    if obs is None:
        return np.frombuffer(raw, dtype=np.complex128)
    vals = np.frombuffer(raw[: 8 * (1 + len(params))], dtype=np.float64)
    return vals[0], vals[1:], np.frombuffer(raw[8 * (1 + len(params)):], dtype=np.complex128)


TOL = {16: 1e-10, 8: 2e-5}
GATE_CODES = {}


@pytest.mark.parametrize("seed", range(16))
@pytest.mark.parametrize("elem_bytes", [16, 8])
def test_random_circuits(emu, tmp_path, seed, elem_bytes):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(2, 12))
    L = int(rng.integers(1, n + 1))
    n_fixed = int(rng.integers(0, min(4, L - 1) + 1)) if L > 1 else 0
    circ = C.random_circuit(n, int(rng.integers(20, 160)), seed)
    psi0 = C.random_state(n, seed)
    got = run_emu(emu, tmp_path, circ, L, n_fixed, None, psi0, elem_bytes)
    ref = S.simulate(circ, None, psi0)
    assert np.linalg.norm(got - ref) <= TOL[elem_bytes]


@pytest.mark.parametrize("elem_bytes", [16, 8])
@pytest.mark.parametrize("n,L", [(10, 7), (12, 9), (11, 11)])
def test_qft_roundtrip_pair_phases(emu, tmp_path, elem_bytes, n, L):
    """QFT and its inverse: controlled phases between register bits fold into the
    following real butterflies (pair phases); the rest become twiddles and slots."""
    circ = C.qft_roundtrip(n)
    psi0 = C.random_state(n, 3)
    got = run_emu(emu, tmp_path, circ, L, min(4, L - 1), None, psi0, elem_bytes)
    assert np.linalg.norm(got - psi0) <= TOL[elem_bytes]
    half = C.Circuit(n, circ.gates[: len(circ.gates) // 2], 0)
    got = run_emu(emu, tmp_path, half, L, min(4, L - 1), None, psi0, elem_bytes)
    assert np.linalg.norm(got - S.simulate(half, None, psi0)) <= TOL[elem_bytes]


@pytest.mark.parametrize("elem_bytes", [16, 8])
@pytest.mark.parametrize("rmax", [2, 3, 4])
def test_parametric_ansatz(emu, tmp_path, elem_bytes, rmax):
    n = 9
    circ = C.hea(n, 4)
    p = C.hea_params(circ.n_params, 7)
    psi0 = C.random_state(n, 7)
    got = run_emu(emu, tmp_path, circ, 7, 3, p, psi0, elem_bytes, rmax)
    assert np.linalg.norm(got - S.simulate(circ, p, psi0)) <= TOL[elem_bytes]


@pytest.mark.parametrize("elem_bytes", [16, 8])
def test_brickwork_config(emu, tmp_path, elem_bytes):
    circ = C.brickwork(11, 10, 1)
    psi0 = C.random_state(11, 1)
    got = run_emu(emu, tmp_path, circ, 8, 4, None, psi0, elem_bytes)
    assert np.linalg.norm(got - S.simulate(circ, None, psi0)) <= TOL[elem_bytes]


def _mixed_ansatz(n, layers, seed):
    """Hardware-efficient layers (parametric RX / RY / RZ, CX / CZ) with fixed gates
    sprinkled in, SWAPs among them (so the adjoint runs in a relabelled layout)."""
    rng = np.random.default_rng(seed)
    gates, p = [], 0
    for _ in range(layers):
        for q in range(n):
            gates.append(C.Gate(("RX", "RY")[int(rng.integers(0, 2))], (q,), p)); p += 1
            gates.append(C.Gate("RZ", (q,), p)); p += 1
        for q in range(n - 1):
            gates.append(C.Gate(("CX", "CZ")[int(rng.integers(0, 2))], (q, q + 1)))
        for _ in range(3):
            k = ("H", "T", "S", "CP", "U3", "SWAP")[int(rng.integers(0, 6))]
            if k in ("CP", "SWAP"):
                a, b = (int(x) for x in rng.choice(n, size=2, replace=False))
                gates.append(C.Gate(k, (a, b), -1, (float(rng.uniform(-3, 3)),) if k == "CP" else ()))
            elif k == "U3":
                gates.append(C.Gate(k, (int(rng.integers(0, n)),), -1, tuple(float(x) for x in rng.uniform(-3, 3, 3))))
            else:
                gates.append(C.Gate(k, (int(rng.integers(0, n)),)))
    return C.Circuit(n, gates, p)


@pytest.mark.parametrize("bind", [False, True])
@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("elem_bytes", [16, 8])
def test_adjoint_gradient(emu, tmp_path, seed, elem_bytes, bind):
    """sv_grad's lowering (parameters bound at lowering) and the batched form's (bound
    dense ops whose matrices are formed from the parameters after packing)."""
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(6, 10))
    L = int(rng.integers(5, n + 1))
    circ = _mixed_ansatz(n, int(rng.integers(1, 4)), seed)
    p = C.hea_params(circ.n_params, seed)
    terms = list(C.tfim(n).terms)
    for _ in range(6):
        c = ["I"] * n
        for q in rng.choice(n, size=int(rng.integers(1, 4)), replace=False):
            c[q] = "XYZ"[int(rng.integers(0, 3))]
        terms.append((float(rng.normal()), "".join(c)))
    obs = C.Observable(n, terms)
    psi0 = C.zero_state(n)
    E, g, back = run_emu(emu, tmp_path, circ, L, min(4, L - 1), p, psi0, elem_bytes,
                         4 if elem_bytes == 8 else 3, obs, bind)
    e_ref = O.expval(S.simulate(circ, p), obs)
    g_ps = GR.parameter_shift(circ, p, obs)
    if elem_bytes == 16:
        assert abs(E - e_ref) <= 1e-10 * max(1.0, abs(e_ref))
        assert np.linalg.norm(g - g_ps) <= 1e-9 * max(1.0, np.linalg.norm(g_ps))
        assert np.linalg.norm(back - psi0) <= 1e-10
    else:
        assert abs(E - e_ref) <= 1e-6 * max(1.0, abs(e_ref))
        assert np.linalg.norm(g - g_ps) <= 1e-4 * np.linalg.norm(g_ps)
        assert np.linalg.norm(back - psi0) <= 1e-4


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("k", [5, 6, 7])
@pytest.mark.parametrize("n,seed", [(8, 1), (11, 2), (14, 3)])
def test_tensor_core_plan(emu, tmp_path, prec, k, n, seed):
    """The tensor-core planner (strict partition, fused unitary, real embedding, hi / lo
    split, 128-byte-swizzled B blob, local / column / global bit roles), decoded and
    applied in FP64 (the state itself unsplit): only the split of the unitary remains,
    about 2^-22 (TF32 pair) or 2^-17 (BF16 pair) relative per element, so 2e-7 (TF32x3)
    and 2e-6 (BF16x3) per fused stage."""
    if n < k + 1:
        pytest.skip("narrower than the stage needs")
    circ = C.brickwork(n, 10, seed)
    psi0 = C.random_state(n, seed)
    nst, got = run_emu(emu, tmp_path, circ, k, 0, None, psi0, 8, prec, gemm=True)
    ref = S.simulate(circ, None, psi0)
    assert nst >= 1
    assert np.linalg.norm(got - ref) <= (2e-7 if prec == 1 else 2e-6) * nst


@pytest.mark.parametrize("case", ["qft", "random_swaps"])
@pytest.mark.parametrize("n,L", [(9, 5), (12, 7), (13, 11)])
def test_fused_output_permutation_lowering(emu, tmp_path, case, n, L):
    """Lowering for a last stage that writes through the final map (Sec. 4.3 reshaping
    fused into the write-back): its tile trades untouched fill bits for the bits that
    become the lowest qubits; the program must still compute the circuit."""
    if case == "qft":
        circ = C.qft(n)
    else:
        circ = C.random_circuit(n, 80, n + L)
        rng = np.random.default_rng(n * L)
        for _ in range(4):
            a, b = (int(x) for x in rng.choice(n, 2, replace=False))
            circ.gates.append(C.Gate("SWAP", (a, b), -1, ()))
    psi0 = C.random_state(n, 9)
    ref = S.simulate(circ, None, psi0)
    got = run_emu(emu, tmp_path, circ, L, min(4, L - 1), None, psi0, 8, fuse=True)
    assert np.linalg.norm(got - ref) <= TOL[8]


@pytest.mark.parametrize("prec,k", [(2, 5), (2, 6), (1, 5)])
@pytest.mark.parametrize("case", ["brick", "qft", "random", "long"])
def test_hierarchical_plan(emu, tmp_path, prec, k, case):
    """Tiles of k + 7 qubits, each stage partitioned again into k-qubit sub-partitions
    applied as split-precision GEMMs (Sec. 4.2's recursive partitioning): the emulated
    operand layouts, splits and products must reproduce the oracle, within the derived
    bound of the sub-partitions' GEMMs (each 3 (K / 8) 2^-23 for the accumulation, K =
    2^(k+1), plus the state split's 2^-16 (BF16x3) / 2^-22 (TF32x3)); two global qubits
    give four tiles per stage."""
    n = k + 9
    circ = {"brick": lambda: C.brickwork(n, 8, 3), "qft": lambda: C.qft(n),
            "random": lambda: C.random_circuit(n, 150, 11),
            "long": lambda: C.Circuit(n, C.random_circuit(12, 700, 3).gates)}[case]()   # > 24 sub-partitions
    psi0 = C.random_state(n, 5)
    ref = S.simulate(circ, None, psi0)
    n_sub, got = run_emu(emu, tmp_path, circ, k + 7, 4, None, psi0, 8, rmax=prec, hier=True)
    bound = n_sub * (3 * (2 ** (k + 1) / 8) * 2.0 ** -23 + (2.0 ** -16 if prec == 2 else 2.0 ** -22))
    err = np.linalg.norm(got - ref)
    assert err <= bound, (n_sub, err, bound)
