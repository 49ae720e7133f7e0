"""Write brick26_oracle.json: reference values of the precision workload at 26 qubits,
computed by the complex128 gate-by-gate oracle only.

Workload: brickwork of depth 24 on 26 qubits (U3 angles uniform in [0, 2pi), seed 3;
CZ on even pairs on even layers, odd pairs on odd layers), applied to the seeded
random state random_state(26, 3) rounded to complex64 (the value a complex64 run
starts from; reading: gate matrices and inputs are rounded once at the boundary).

Stored: 64 sampled output amplitudes (indices drawn with default_rng(26)), <Z_q> for
every qubit, and ||psi||^2.  Runs for tens of minutes on one CPU core:

    python tests/golden/make_brick26_oracle.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import circuits as C  # noqa: E402  (seeded generators: data only)
from oracle import observables as O  # noqa: E402
from oracle import statevector as S  # noqa: E402

N, DEPTH, SEED, SAMPLE_SEED, N_SAMPLES = 26, 24, 3, 26, 64


def main(out=os.path.join(HERE, "brick26_oracle.json")):
    t0 = time.time()
    circ = C.brickwork(N, DEPTH, SEED)
    psi0 = C.random_state(N, SEED).astype(np.complex64).astype(np.complex128)
    psi = S.simulate(circ, None, psi0)
    idx = sorted(int(i) for i in np.random.default_rng(SAMPLE_SEED).choice(1 << N, N_SAMPLES, replace=False))
    zq = []
    for q in range(N):
        s = ["I"] * N
        s[q] = "Z"
        zq.append(float(O.expval(psi, C.Observable(N, [(1.0, "".join(s))]))))
    rec = {
        "source": "precision workload (brickwork of depth 24, U3 + CZ) at 26 qubits; the exact result is the "
                  "product of the gates in circuit order (Sec. 4.1-4.2: partitioning reorders nothing), "
                  "computed by the complex128 gate-by-gate oracle",
        "script": "tests/golden/make_brick26_oracle.py",
        "n_qubits": N, "depth": DEPTH, "circuit_seed": SEED,
        "input": "circuits.random_state(26, 3) rounded to complex64",
        "sample_seed": SAMPLE_SEED,
        "indices": idx,
        "amplitudes": [[float(psi[i].real), float(psi[i].imag)] for i in idx],
        "z_expectations": zq,
        "norm2": float(np.vdot(psi, psi).real),
        "oracle_seconds": round(time.time() - t0, 1),
    }
    with open(out, "w") as f:
        json.dump(rec, f, indent=1)
    print(f"wrote {out} in {rec['oracle_seconds']} s")


if __name__ == "__main__":
    main()
