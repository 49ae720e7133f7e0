"""GPU parity on the paper's other benchmark families (Sec. 5.1: AE, DJ, GHZ, Ising,
QFT, QPE, SU2, VQC) and on a circuit read from OpenQASM text: the CUDA path through
the C ABI against the CPU oracle, element by element (complex64 2e-5, complex128
1e-12 in the 2-norm), and adjoint gradients of the parametric families against the
oracle's parameter-shift gradient (1e-4 relative)."""
import numpy as np
import pytest

import circuits as C
from oracle import gradients as GR
from oracle import observables as O
from oracle import statevector as S

pytestmark = pytest.mark.gpu

TOL = {0: 2e-5, 1: 1e-12}


@pytest.fixture(scope="module")
def sv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__ as ge
    ge.build()
    import paper_2509_14098_gb300 as pkg
    return pkg


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("name", sorted(C.FAMILIES))
def test_family_vs_oracle(sv, name, dtype):
    n = 14
    c = C.FAMILIES[name](n)
    p = C.hea_params(c.n_params, 5) if c.n_params else None
    psi0 = C.random_state(n, 6)
    st = sv.StateVector(n, dtype)
    st.set_host(psi0)
    st.run(sv.Plan(c, 9), p)
    got = st.get_host().astype(np.complex128)
    ref = S.simulate(c, p, psi0)
    assert np.linalg.norm(got - ref) <= TOL[dtype], name


@pytest.mark.parametrize("name", ["su2", "vqc"])
def test_family_gradients(sv, name):
    n = 10
    c = C.FAMILIES[name](n)
    p = C.hea_params(c.n_params, 7)
    obs = C.tfim(n)
    e, g = sv.StateVector(n).grad(sv.Plan(c, 7), p, obs)
    assert abs(e - O.expval(S.simulate(c, p), obs)) <= 1e-6 * max(1.0, abs(e))
    g_ps = GR.parameter_shift(c, p, obs)
    assert np.linalg.norm(g - g_ps) <= 1e-4 * np.linalg.norm(g_ps)


def test_qasm_circuit_on_gpu(sv):
    n = 12
    src = C.to_qasm(C.qpe(n, 2)) + "rzz(0.37) q[3],q[9];\nu2(0.1,0.2) q[5];\n"
    qc = sv.parse_qasm(src)
    ref_c = C.Circuit(n, [C.Gate(g.kind, g.qubits, -1, g.angles) for g in qc.gates])
    st = sv.StateVector(n)
    st.run(sv.Plan(qc, 8))
    assert np.linalg.norm(st.get_host().astype(np.complex128) - S.simulate(ref_c)) <= 2e-5
