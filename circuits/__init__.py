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
