"""Seeded synthetic workloads shared by the oracle and the GPU path.

This module holds data only: gate lists (kind, qubits, parameter slot, fixed
angles), parameter vectors, initial states and Pauli observables.  It contains
none of the method's arithmetic (no gate matrices, no state updates, no
partitioning), so both the CPU oracle and the CUDA path may import it without
sharing any computation.

Qubit convention: qubit q is bit q of the amplitude index (little-endian).
A two-qubit gate lists its qubits as (q0, q1); for controlled gates q0 is the
control and q1 the target.

Workload recipes follow the circuit families the paper evaluates (QFT, random
brickwork / SU2-style, variational ansatz; Sec. 5.1) with the sizes of the
benchmark configurations below.  The paper's suites (MQTBench, QASMBench) are
not available, so these seeded generators stand in for them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Gate kinds understood by both sides.  Diagonal kinds carry no dense action.
KINDS = ("H", "X", "Y", "Z", "S", "SDG", "T", "TDG", "RX", "RY", "RZ", "P",
         "U3", "CX", "CY", "CZ", "CP", "SWAP")
ONE_QUBIT = {"H", "X", "Y", "Z", "S", "SDG", "T", "TDG", "RX", "RY", "RZ", "P", "U3"}
TWO_QUBIT = {"CX", "CY", "CZ", "CP", "SWAP"}
PARAMETRIC = {"RX", "RY", "RZ", "P", "CP"}   # gates whose single angle may be a parameter slot
N_ANGLES = {"RX": 1, "RY": 1, "RZ": 1, "P": 1, "CP": 1, "U3": 3}


@dataclass(frozen=True)
class Gate:
    kind: str
    qubits: Tuple[int, ...]
    param: int = -1                     # index into the parameter vector, -1 = fixed angles
    angles: Tuple[float, ...] = ()      # fixed angles (used when param == -1)

    def __post_init__(self):
        if self.kind not in KINDS:
            raise ValueError(f"unknown gate kind {self.kind}")
        nq = 1 if self.kind in ONE_QUBIT else 2
        if len(self.qubits) != nq:
            raise ValueError(f"{self.kind} takes {nq} qubits")
        if nq == 2 and self.qubits[0] == self.qubits[1]:
            raise ValueError("two-qubit gate on a single qubit")
        if self.param >= 0 and self.kind not in PARAMETRIC:
            raise ValueError(f"{self.kind} cannot be parametric")


@dataclass
class Circuit:
    n_qubits: int
    gates: List[Gate] = field(default_factory=list)
    n_params: int = 0
    name: str = ""

    def __len__(self):
        return len(self.gates)

    def angles_of(self, g: Gate, params: Optional[Sequence[float]]) -> Tuple[float, ...]:
        """The angles a gate uses: its parameter slot when it has one."""
        if g.param >= 0:
            if params is None:
                raise ValueError("circuit has parameters but none were given")
            return (float(params[g.param]),)
        return tuple(g.angles)


# ----------------------------------------------------------------------------
# Generators
# ----------------------------------------------------------------------------

def ghz(n: int) -> Circuit:
    """H on qubit 0 then a CX chain; n=3 is the paper's worked example (Sec. 4.1)."""
    gates = [Gate("H", (0,))] + [Gate("CX", (q, q + 1)) for q in range(n - 1)]
    return Circuit(n, gates, 0, f"ghz{n}")


def qft(n: int) -> Circuit:
    """Little-endian QFT: for j = n-1..0: H(j), then CP(pi/2^(j-m)) on (m, j) for m = j-1..0;
    then the bit-reversal SWAPs.  n(n-1)/2 controlled phases with angles 2*pi/2^k."""
    gates: List[Gate] = []
    for j in range(n - 1, -1, -1):
        gates.append(Gate("H", (j,)))
        for m in range(j - 1, -1, -1):
            gates.append(Gate("CP", (m, j), -1, (math.pi / (1 << (j - m)),)))
    for q in range(n // 2):
        gates.append(Gate("SWAP", (q, n - 1 - q)))
    return Circuit(n, gates, 0, f"qft{n}")


_DAGGER_KIND = {"S": "SDG", "SDG": "S", "T": "TDG", "TDG": "T"}


def inverse(c: Circuit) -> Circuit:
    """Reverse gate order and conjugate each gate (fixed-angle gates only: the
    inverse of a rotation negates its angle; U3(t,p,l)^-1 = U3(-t,-l,-p))."""
    out: List[Gate] = []
    for g in reversed(c.gates):
        if g.param >= 0:
            raise ValueError("inverse() needs fixed angles")
        k = _DAGGER_KIND.get(g.kind, g.kind)
        if g.kind == "U3":
            t, p, l = g.angles
            out.append(Gate("U3", g.qubits, -1, (-t, -l, -p)))
        elif g.kind in ("RX", "RY", "RZ", "P", "CP"):
            out.append(Gate(g.kind, g.qubits, -1, (-g.angles[0],)))
        else:
            out.append(Gate(k, g.qubits, -1, ()))
    return Circuit(c.n_qubits, out, 0, c.name + "_inv")


def concat(a: Circuit, b: Circuit) -> Circuit:
    if a.n_qubits != b.n_qubits or a.n_params or b.n_params:
        raise ValueError("concat needs equal widths and fixed angles")
    return Circuit(a.n_qubits, list(a.gates) + list(b.gates), 0, a.name + "+" + b.name)


def qft_roundtrip(n: int) -> Circuit:
    """QFT followed by its inverse (identity overall)."""
    return concat(qft(n), inverse(qft(n)))


def brickwork(n: int, layers: int, seed: int) -> Circuit:
    """Layer l: U3(theta, phi, lambda) on every qubit with angles uniform in [0, 2pi),
    drawn in gate order (theta, phi, lambda per gate), then CZ(q, q+1) for q = l mod 2,
    l mod 2 + 2, ... (even pairs on even layers, odd pairs on odd layers)."""
    rng = np.random.default_rng(seed)
    gates: List[Gate] = []
    for layer in range(layers):
        for q in range(n):
            a = rng.uniform(0.0, 2.0 * math.pi, size=3)
            gates.append(Gate("U3", (q,), -1, (float(a[0]), float(a[1]), float(a[2]))))
        for q in range(layer % 2, n - 1, 2):
            gates.append(Gate("CZ", (q, q + 1)))
    return Circuit(n, gates, 0, f"brick{n}x{layers}")


def hea(n: int, layers: int) -> Circuit:
    """Hardware-efficient ansatz: per layer RY(q) on all q, RZ(q) on all q, then the
    CNOT ladder CX(q, q+1), q = 0..n-2.  Parameters are layer-major, RY before RZ,
    qubit ascending: slot = layer*2n + (0 for RY, n for RZ) + q."""
    gates: List[Gate] = []
    for layer in range(layers):
        base = layer * 2 * n
        for q in range(n):
            gates.append(Gate("RY", (q,), base + q))
        for q in range(n):
            gates.append(Gate("RZ", (q,), base + n + q))
        for q in range(n - 1):
            gates.append(Gate("CX", (q, q + 1)))
    return Circuit(n, gates, 2 * n * layers, f"hea{n}x{layers}")


def hea_params(n_params: int, seed: int, rng: Optional[np.random.Generator] = None) -> np.ndarray:
    """Parameters uniform in [-pi, pi)."""
    rng = rng if rng is not None else np.random.default_rng(seed)
    return rng.uniform(-math.pi, math.pi, size=n_params)


def random_circuit(n: int, n_gates: int, seed: int, kinds: Sequence[str] = KINDS) -> Circuit:
    """Random gate list over the given kinds (fixed angles), for property tests."""
    rng = np.random.default_rng(seed)
    gates: List[Gate] = []
    for _ in range(n_gates):
        k = str(rng.choice(list(kinds)))
        if k in TWO_QUBIT:
            if n < 2:
                continue
            a, b = rng.choice(n, size=2, replace=False)
            qs = (int(a), int(b))
        else:
            qs = (int(rng.integers(n)),)
        na = N_ANGLES.get(k, 0)
        ang = tuple(float(x) for x in rng.uniform(-math.pi, math.pi, size=na))
        gates.append(Gate(k, qs, -1, ang))
    return Circuit(n, gates, 0, f"rand{n}x{n_gates}")


def batch_spec(count: int, seed: int, n_lo: int = 10, n_hi: int = 20, layers: int = 6):
    """Heterogeneous batch: draw every qubit count first (uniform in [n_lo, n_hi]),
    then each circuit's parameters in order.  Returns [(Circuit, params)]."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    out = []
    for n in ns:
        c = hea(int(n), layers)
        out.append((c, hea_params(c.n_params, 0, rng)))
    return out


# ----------------------------------------------------------------------------
# The paper's other benchmark families (Sec. 5.1: AE, DJ, GHZ, Ising, QFT, QPE,
# SU2, VQC), as seeded generators written from each algorithm's definition.  They
# stand in for the MQTBench / QASMBench circuit files, which are not available.
# ----------------------------------------------------------------------------

def _iqft_on(qubits: Sequence[int]) -> List[Gate]:
    """Inverse QFT (with the final swaps) on the listed qubits, qubits[0] the least
    significant."""
    m = len(qubits)
    return [Gate(g.kind, tuple(qubits[q] for q in g.qubits), g.param, g.angles) for g in inverse(qft(m)).gates]


def qpe(n: int, seed: int = 0, exact: bool = False) -> Circuit:
    """Phase estimation of P(2 pi phi) on qubit n-1 (prepared in |1>) with n-1
    counting qubits 0..n-2: H on the counting register, CP(2 pi phi 2^k) from counting
    qubit k, then the inverse QFT on the counting register.  phi is drawn from
    default_rng(seed) (exact=True: a multiple of 2^-(n-1), which the circuit resolves
    to a basis state)."""
    m = n - 1
    rng = np.random.default_rng(seed)
    phi = int(rng.integers(1 << m)) / (1 << m) if exact else float(rng.uniform(0.0, 1.0))
    gates = [Gate("X", (n - 1,))] + [Gate("H", (q,)) for q in range(m)]
    for k in range(m):
        gates.append(Gate("CP", (k, n - 1), -1, (2.0 * math.pi * phi * (1 << k) % (2.0 * math.pi),)))
    gates += _iqft_on(list(range(m)))
    c = Circuit(n, gates, 0, f"qpe{n}")
    c.phase = phi
    return c


def dj(n: int, seed: int = 0) -> Circuit:
    """Deutsch-Jozsa with a balanced oracle on n-1 input qubits and ancilla n-1:
    X(anc); H on all; oracle f(x) = x.b xor parity of the X-mask (X on the masked
    inputs, CX from every input to the ancilla, X again); H on the inputs."""
    m = n - 1
    rng = np.random.default_rng(seed)
    xmask = rng.integers(0, 2, size=m)
    gates = [Gate("X", (m,))] + [Gate("H", (q,)) for q in range(n)]
    gates += [Gate("X", (q,)) for q in range(m) if xmask[q]]
    gates += [Gate("CX", (q, m)) for q in range(m)]
    gates += [Gate("X", (q,)) for q in range(m) if xmask[q]]
    gates += [Gate("H", (q,)) for q in range(m)]
    return Circuit(n, gates, 0, f"dj{n}")


def su2(n: int, reps: int = 3) -> Circuit:
    """EfficientSU2-style ansatz: per repetition RY and RZ on every qubit and a linear
    CX chain, then a final RY / RZ layer.  Parameters: layer-major, RY before RZ."""
    gates: List[Gate] = []
    slot = 0
    for r in range(reps + 1):
        for kind in ("RY", "RZ"):
            for q in range(n):
                gates.append(Gate(kind, (q,), slot))
                slot += 1
        if r < reps:
            gates += [Gate("CX", (q, q + 1)) for q in range(n - 1)]
    return Circuit(n, gates, slot, f"su2_{n}x{reps}")


def ising(n: int, steps: int = 4, J: float = 1.0, h: float = 0.7, dt: float = 0.1) -> Circuit:
    """First-order Trotter steps of the transverse-field Ising chain: per step
    exp(-i J dt Z_q Z_{q+1}) as CX(q, q+1) RZ(2 J dt)(q+1) CX(q, q+1) on every bond,
    then RX(2 h dt) on every qubit."""
    gates: List[Gate] = []
    for _ in range(steps):
        for q in range(n - 1):
            gates += [Gate("CX", (q, q + 1)), Gate("RZ", (q + 1,), -1, (2 * J * dt,)), Gate("CX", (q, q + 1))]
        gates += [Gate("RX", (q,), -1, (2 * h * dt,)) for q in range(n)]
    return Circuit(n, gates, 0, f"ising{n}x{steps}")


def vqc(n: int, reps: int = 2, seed: int = 0) -> Circuit:
    """Variational classifier: a second-order Pauli-Z feature map of seeded data x
    (H, P(2 x_q), and per neighbour pair CX . P(2 (pi - x_q)(pi - x_{q+1})) . CX),
    then a real-amplitudes ansatz (RY layers and CX chains, parameters layer-major)."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 2.0 * math.pi, size=n)
    gates = [Gate("H", (q,)) for q in range(n)]
    gates += [Gate("P", (q,), -1, (2.0 * float(x[q]),)) for q in range(n)]
    for q in range(n - 1):
        a = 2.0 * (math.pi - float(x[q])) * (math.pi - float(x[q + 1]))
        gates += [Gate("CX", (q, q + 1)), Gate("P", (q + 1,), -1, (a,)), Gate("CX", (q, q + 1))]
    slot = 0
    for r in range(reps + 1):
        for q in range(n):
            gates.append(Gate("RY", (q,), slot))
            slot += 1
        if r < reps:
            gates += [Gate("CX", (q, q + 1)) for q in range(n - 1)]
    return Circuit(n, gates, slot, f"vqc{n}x{reps}")


def ae(n: int, p: float = 0.2) -> Circuit:
    """Amplitude estimation of a = p for A = RY(theta_p) on objective qubit n-1
    (sin^2(theta_p / 2) = p), with n-1 counting qubits: A, H on the counting register,
    controlled powers Q^(2^k) of the Grover operator (for one objective qubit, Q is
    RY(2 theta_p); controlled RY(t) is emitted as RY(t/2) CX RY(-t/2) CX on the
    target), then the inverse QFT on the counting register."""
    m = n - 1
    tgt = n - 1
    theta = 2.0 * math.asin(math.sqrt(p))
    gates = [Gate("RY", (tgt,), -1, (theta,))] + [Gate("H", (q,)) for q in range(m)]
    for k in range(m):
        t = (2.0 * theta * (1 << k)) % (4.0 * math.pi)
        gates += [Gate("RY", (tgt,), -1, (t / 2,)), Gate("CX", (k, tgt)),
                  Gate("RY", (tgt,), -1, (-t / 2,)), Gate("CX", (k, tgt))]
    gates += _iqft_on(list(range(m)))
    return Circuit(n, gates, 0, f"ae{n}")


# name -> (generator of width n, number of parameters or 0)
FAMILIES = {
    "ae": lambda n: ae(n),
    "dj": lambda n: dj(n, 1),
    "ghz": lambda n: ghz(n),
    "ising": lambda n: ising(n, 4),
    "qft": lambda n: qft(n),
    "qpe": lambda n: qpe(n, 1),
    "su2": lambda n: su2(n, 3),
    "vqc": lambda n: vqc(n, 2, 1),
}


def to_qasm(c: Circuit, params: Optional[Sequence[float]] = None) -> str:
    """OpenQASM 2.0 text of a circuit (parameters substituted; angles in full
    precision)."""
    names = {"H": "h", "X": "x", "Y": "y", "Z": "z", "S": "s", "SDG": "sdg", "T": "t", "TDG": "tdg",
             "RX": "rx", "RY": "ry", "RZ": "rz", "P": "p", "U3": "u3", "CX": "cx", "CY": "cy", "CZ": "cz",
             "CP": "cp", "SWAP": "swap"}
    out = ["OPENQASM 2.0;", 'include "qelib1.inc";', f"qreg q[{c.n_qubits}];", f"creg c[{c.n_qubits}];"]
    for g in c.gates:
        ang = c.angles_of(g, params)
        a = "(" + ",".join(repr(float(x)) for x in ang) + ")" if ang else ""
        out.append(f"{names[g.kind]}{a} " + ",".join(f"q[{q}]" for q in g.qubits) + ";")
    out.append("measure q -> c;")
    return "\n".join(out) + "\n"


# ----------------------------------------------------------------------------
# States and observables (data)
# ----------------------------------------------------------------------------

def random_state(n: int, seed: int) -> np.ndarray:
    """i.i.d. N(0,1) real and imaginary parts, normalised, complex128."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return v / np.linalg.norm(v)


def zero_state(n: int) -> np.ndarray:
    v = np.zeros(1 << n, dtype=np.complex128)
    v[0] = 1.0
    return v


@dataclass
class Observable:
    """Sum of Pauli strings: terms[i] = (coeff, string) where string[q] in 'IXYZ'
    is the Pauli acting on qubit q."""
    n_qubits: int
    terms: List[Tuple[float, str]]


def tfim(n: int, hx: float = 0.7) -> Observable:
    """Open-chain transverse-field Ising: sum_i Z_i Z_{i+1} + hx * sum_i X_i."""
    terms = []
    for i in range(n - 1):
        s = ["I"] * n
        s[i] = s[i + 1] = "Z"
        terms.append((1.0, "".join(s)))
    for i in range(n):
        s = ["I"] * n
        s[i] = "X"
        terms.append((hx, "".join(s)))
    return Observable(n, terms)


def zz_chain(n: int) -> Observable:
    """Open-chain sum_i Z_i Z_{i+1}."""
    return Observable(n, tfim(n, 0.0).terms[: n - 1])


# Benchmark workloads (sizes of the five configurations)
def workload(name: str):
    if name == "brick16":
        return brickwork(16, 20, 1), None, 10
    if name == "qft30":
        return qft_roundtrip(30), None, 11
    if name == "brick32":
        return brickwork(32, 24, 3), None, 11
    if name == "hea28":
        c = hea(28, 10)
        return c, hea_params(c.n_params, 4), 10
    raise KeyError(name)
