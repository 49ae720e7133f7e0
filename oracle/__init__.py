"""CPU oracle — TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct complex128 state-vector simulator and a plain
Python version of the closeness-centrality partitioner, written from the paper.
Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
legs may import it.  The GPU library never imports, links or calls anything here,
and nothing here imports the GPU library: the two share only the seeded input
generators in ``circuits``.

Modules
  gates        gate matrices in FP64 from their formulas (Sec. 3.1)
  statevector  gates applied one at a time, original order, no partitioning (Sec. 3.2, Eq. for xi)
  dense        brute-force dense 2^n x 2^n Kronecker unitaries for small n (Sec. 3.1, G_H = H (x) I (x) I)
  observables  Pauli-sum expectation values
  gradients    central finite differences and the parameter-shift rule
  partition    contraction DAG, critical-path levels, exact closeness centrality and
               the forward frontier partitioner (Sec. 4.1-4.2), plus a validator
"""
