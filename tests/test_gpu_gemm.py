"""Split-precision tensor-core stages (tcgen05) against the complex128 oracle.

Each partition (no exemptions, fusion width k) is one dense unitary applied as a GEMM
with three tensor-core products (hi*hi + lo*hi + hi*lo) accumulated in FP32 in tensor
memory.  Bound: the split keeps ~21 (TF32x3) or ~16 (BF16x3) significant bits per
product, but each output element of a fused stage is accumulated over K = 2^(k+1)
terms in about 3 K / 8 tensor-core accumulation steps whose FP32 additions carry no
IEEE rounding guarantee, i.e. up to ~3 (K / 8) 2^-23 relative per stage (~1e-5 at
K = 256).  The tolerance is therefore 2e-5 per fused stage, accumulated over the stages,
for both precisions.
"""
import numpy as np
import pytest

import circuits as C
from oracle import statevector as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__ as ge
    ge.build()
    import paper_2509_14098_gb300 as pkg
    return pkg


def _run(sv, circ, k, prec, psi0):
    plan = sv.Plan(circ, k, gemm=True)
    st = sv.StateVector(circ.n_qubits)
    st.set_host(psi0)
    st.run(plan, None, prec)
    return st.get_host().astype(np.complex128), len(plan.stages())


@pytest.mark.parametrize("k", [5, 6, 7])
@pytest.mark.parametrize("prec", [1, 2])
def test_brickwork_gemm(sv, k, prec):
    n = 16
    circ = C.brickwork(n, 12, 3)
    psi0 = C.random_state(n, 3)
    got, nst = _run(sv, circ, k, prec, psi0)
    ref = S.simulate(circ, None, psi0)
    err = float(np.linalg.norm(got - ref))
    print(f"brick16 k={k} prec={prec} stages={nst} err={err:.3e}")
    bound = 2e-5 * nst
    assert err <= bound, (err, bound)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("prec", [1, 2])
def test_random_circuits_gemm(sv, seed, prec):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(11, 15))
    k = int(rng.integers(5, 8))
    circ = C.random_circuit(n, int(rng.integers(40, 200)), seed)
    psi0 = C.random_state(n, seed)
    got, nst = _run(sv, circ, k, prec, psi0)
    ref = S.simulate(circ, None, psi0)
    err = float(np.linalg.norm(got - ref))
    print(f"random n={n} k={k} prec={prec} stages={nst} err={err:.3e}")
    bound = 2e-5 * nst
    assert err <= bound, (err, bound)


def test_gemm_plan_on_cuda_cores(sv):
    n = 14
    circ = C.brickwork(n, 8, 5)
    psi0 = C.random_state(n, 5)
    got, _ = _run(sv, circ, 6, 0, psi0)
    assert np.linalg.norm(got - S.simulate(circ, None, psi0)) <= 2e-5


def test_gemm_errors(sv):
    from paper_2509_14098_gb300 import _native as N
    circ = C.brickwork(12, 2, 1)
    with pytest.raises(sv.SvError) as e:
        sv.StateVector(12).run(sv.Plan(circ, 6), None, 1)     # not a tensor-core plan
    assert e.value.status == N.SV_ERR_UNSUPPORTED
    with pytest.raises(sv.SvError):
        sv.Plan(circ, 8, gemm=True)


@pytest.mark.parametrize("k", [5, 6, 7])
@pytest.mark.parametrize("prec", [1, 2])
def test_brick20_vs_complex128(sv, k, prec):
    """A wider state (many tiles per stage, k = 7 streams its B operand) against the
    complex128 CUDA-core run of the same circuit and input."""
    n = 20
    circ = C.brickwork(n, 24, 3)
    psi0 = C.random_state(n, 7)
    ref = sv.StateVector(n, sv.SV_C128)
    ref.set_host(psi0)
    ref.run(sv.Plan(circ, 11))
    r = ref.get_host()
    got, nst = _run(sv, circ, k, prec, psi0.astype(np.complex64))
    err = float(np.linalg.norm(got - r))
    print(f"brick20 k={k} prec={prec} stages={nst} err={err:.3e}")
    bound = 2e-5 * nst
    assert err <= bound, (err, bound)
