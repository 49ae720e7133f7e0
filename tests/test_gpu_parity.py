"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by
element, at sizes spanning several tiles and ragged stage shapes.

Tolerances (from the target): ||psi - psi_ref||_2 <= 2e-5 (complex64),
<= 1e-12 (complex128); expectation values within 1e-6 relative (max(|E|, 1));
gradients within 1e-4 relative of the reference gradient (2-norm).
"""
import math

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


def run_gpu(sv, circ, L, psi0=None, dtype=0, params=None, n_fixed=None):
    plan = sv.Plan(circ, L, n_fixed)
    st = sv.StateVector(circ.n_qubits, dtype)
    if psi0 is not None:
        st.set_host(psi0)
    st.run(plan, params)
    return st.get_host().astype(np.complex128), st, plan


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("seed", range(10))
def test_random_circuits(sv, seed, dtype):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(3, 15))
    L = int(rng.integers(max(1, min(n, 5)), min(n, 13) + 1))
    c = C.random_circuit(n, int(rng.integers(20, 200)), seed)
    psi0 = C.random_state(n, seed)
    nf = None if seed % 3 else int(rng.integers(0, 4))
    got, _, _ = run_gpu(sv, c, L, psi0, dtype, n_fixed=nf)
    ref = S.simulate(c, None, psi0)
    assert np.linalg.norm(got - ref) <= TOL[dtype], (n, L)


def test_brick16_config(sv):
    c, _, L = C.workload("brick16")
    got, st, plan = run_gpu(sv, c, L)
    ref = S.simulate(c)
    assert np.linalg.norm(got - ref) <= 2e-5
    assert abs(st.norm() - 1) < 1e-6


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n,L", [(6, 4), (10, 6), (14, 11), (17, 11), (18, 13)])
def test_qft_matches_oracle_and_fft(sv, n, L, dtype):
    psi0 = C.random_state(n, 2)
    got, st, _ = run_gpu(sv, C.qft(n), L, psi0, dtype)
    ref = S.simulate(C.qft(n), None, psi0)
    assert np.linalg.norm(got - ref) <= TOL[dtype]
    assert np.linalg.norm(got - np.fft.ifft(psi0, norm="ortho")) <= TOL[dtype]
    # the bit reversal left by the SWAPs: complex64 stages write it in the last stage's
    # write-back, complex128 runs one permutation sweep
    assert st.run_info()["permutation_sweeps"] == (0 if dtype == 0 else 1)


@pytest.mark.parametrize("n,L", [(12, 6), (16, 11)])
def test_fused_permutation_on_an_owned_state(sv, n, L):
    """A handle that owns its state (sv_create with no buffer): the permuted last stage
    leaves the state in the handle's second buffer, which sv_info then reports."""
    import ctypes
    from paper_2509_14098_gb300 import _native as N
    psi0 = C.random_state(n, 4).astype(np.complex64)
    h = ctypes.c_void_p()
    N.check(N.lib.sv_create(n, 0, None, None, ctypes.byref(h)))
    try:
        N.check(N.lib.sv_set_state_host(h, psi0.ctypes.data_as(ctypes.c_void_p)))
        plan = sv.Plan(C.qft(n), L)
        N.check(N.lib.sv_run(h, plan.handle, None, 0))
        out = np.empty_like(psi0)
        N.check(N.lib.sv_get_state_host(h, out.ctypes.data_as(ctypes.c_void_p)))
        ref = S.simulate(C.qft(n), None, psi0.astype(np.complex128))
        assert np.linalg.norm(out - ref) <= 2e-5
        info = N.sv_run_info()
        N.check(N.lib.sv_last_run_info(h, ctypes.byref(info)))
        assert info.permutation_sweeps == 0
        # a second run (the inverse transform) from the moved state restores the input
        inv = sv.Plan(C.inverse(C.qft(n)), L)
        N.check(N.lib.sv_run(h, inv.handle, None, 0))
        N.check(N.lib.sv_get_state_host(h, out.ctypes.data_as(ctypes.c_void_p)))
        assert np.linalg.norm(out - psi0) <= 4e-5
    finally:
        N.lib.sv_destroy(h)


@pytest.mark.parametrize("dtype", [0, 1])
def test_qft_roundtrip_identity(sv, dtype):
    n = 20
    psi0 = C.random_state(n, 2)
    got, st, _ = run_gpu(sv, C.qft_roundtrip(n), 11, psi0, dtype)
    assert np.linalg.norm(got - psi0) <= TOL[dtype]
    info = st.run_info()
    assert info["permutation_sweeps"] == 0               # the two relabels cancel


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("seed", range(4))
def test_permutation_sweep(sv, seed, dtype):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(4, 19))
    perm = [int(x) for x in rng.permutation(n)]
    psi0 = C.random_state(n, seed)
    st = sv.StateVector(n, dtype)
    st.set_host(psi0)
    st.permute(perm)
    got = st.get_host()
    assert np.array_equal(got, S.permute_qubits(psi0, n, perm).astype(got.dtype))   # a pure data move: bit-exact


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("owned", [False, True])
def test_permutation_sweep_many_tiles(sv, dtype, owned):
    """Widths at which every persistent CTA of the permutation sweep takes several tiles
    (both tile buffers in use, a new global offset per tile): the bit reversal, then a
    random permutation of the result, on a borrowed buffer (the result is copied back)
    and on a handle that owns its state (the result buffer becomes the state)."""
    import ctypes
    from paper_2509_14098_gb300 import _native as N
    n = 24 if dtype == 0 else 23
    npdt = np.complex64 if dtype == 0 else np.complex128
    psi0 = C.random_state(n, 11).astype(npdt)
    rev = list(range(n))[::-1]
    perm = [int(x) for x in np.random.default_rng(11).permutation(n)]
    want = S.permute_qubits(S.permute_qubits(psi0, n, rev), n, perm)
    out = np.empty_like(psi0)
    if owned:
        h = ctypes.c_void_p()
        N.check(N.lib.sv_create(n, dtype, None, None, ctypes.byref(h)))
        try:
            N.check(N.lib.sv_set_state_host(h, psi0.ctypes.data_as(ctypes.c_void_p)))
            for p in (rev, perm):
                N.check(N.lib.sv_permute(h, (ctypes.c_uint32 * n)(*p)))
            N.check(N.lib.sv_get_state_host(h, out.ctypes.data_as(ctypes.c_void_p)))
        finally:
            N.lib.sv_destroy(h)
    else:
        st = sv.StateVector(n, dtype)
        st.set_host(psi0)
        st.permute(rev)
        st.permute(perm)
        out = st.get_host()
    assert np.array_equal(out, want)   # a pure data move: bit-exact


@pytest.mark.parametrize("dtype", [0, 1])
def test_norm_and_expval(sv, dtype):
    n = 13
    psi = C.random_state(n, 7)
    st = sv.StateVector(n, dtype)
    st.set_host(psi)
    rng = np.random.default_rng(3)
    terms = [(float(rng.normal()), "".join(rng.choice(list("IXYZ"), size=n))) for _ in range(25)]
    terms += C.tfim(n).terms
    obs = C.Observable(n, terms)
    e_ref = O.expval(psi, obs)
    tol = 1e-6 * max(1.0, abs(e_ref)) if dtype == 0 else 1e-11
    assert abs(st.expval(obs) - e_ref) <= tol
    assert abs(st.norm() - 1.0) <= (1e-6 if dtype == 0 else 1e-12)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_tiny_states(sv, n):
    c = C.random_circuit(n, 30, n)
    psi0 = C.random_state(n, n)
    got, st, _ = run_gpu(sv, c, n, psi0)
    assert np.linalg.norm(got - S.simulate(c, None, psi0)) <= 2e-5
    obs = C.tfim(n)
    assert abs(st.expval(obs) - O.expval(got, obs)) <= 1e-6 * max(1, abs(O.expval(got, obs)))


@pytest.mark.parametrize("dtype", [0, 1])
def test_degenerate_circuits(sv, dtype):
    """The method's degenerate cases: an empty circuit leaves the state bit-exact; a
    circuit of diagonal gates only (every gate exempt, one stage with no dense op); a
    circuit of SWAPs only (pure relabels: the state moves by the final qubit map only,
    bit-exact); a budget L >= n (the whole state is one tile)."""
    n = 14
    psi0 = C.random_state(n, 21)
    npdt = np.complex64 if dtype == 0 else np.complex128
    tol = TOL[dtype]
    got, _, _ = run_gpu(sv, C.Circuit(n, []), 11, psi0, dtype)
    assert np.array_equal(got, psi0.astype(npdt).astype(np.complex128))
    rng = np.random.default_rng(21)
    diag = C.Circuit(n, [C.Gate(k, tuple(int(q) for q in rng.choice(n, 2 if k in ("CZ", "CP") else 1, replace=False)), -1,
                                (float(rng.uniform(0, 2 * np.pi)),) if k in ("RZ", "P", "CP") else ())
                         for k in map(str, rng.choice(["Z", "S", "T", "SDG", "TDG", "RZ", "P", "CZ", "CP"], 60))])
    got, _, _ = run_gpu(sv, diag, 11, psi0, dtype)
    assert np.linalg.norm(got - S.simulate(diag, None, psi0)) <= tol
    swaps = C.Circuit(n, [C.Gate("SWAP", tuple(int(q) for q in rng.choice(n, 2, replace=False))) for _ in range(9)])
    got, st, _ = run_gpu(sv, swaps, 11, psi0, dtype)
    assert np.array_equal(got, S.simulate(swaps, None, psi0.astype(npdt).astype(np.complex128)))
    assert st.run_info()["stage_sweeps"] + st.run_info()["permutation_sweeps"] <= 2
    n1 = 14 if dtype == 0 else 13   # the widest tile of the dtype (128 KB / 128 KB)
    c = C.random_circuit(n1, 120, 5)
    psi1 = C.random_state(n1, 22)
    got, st, _ = run_gpu(sv, c, n1, psi1, dtype)
    assert np.linalg.norm(got - S.simulate(c, None, psi1)) <= tol
    assert st.run_info()["stage_sweeps"] == 1


@pytest.fixture(scope="module")
def hea12_reference():
    """The differentiation workload at oracle size (12 qubits, 10 layers, 240
    parameters): <H> and its gradient by parameter shift and by central finite
    differences, both on the oracle."""
    c = C.hea(12, 10)
    p = C.hea_params(c.n_params, 4)
    obs = C.tfim(12)
    e_ref = O.expval(S.simulate(c, p), obs)
    return c, p, obs, e_ref, GR.parameter_shift(c, p, obs), GR.finite_difference(c, p, obs)


@pytest.mark.parametrize("dtype", [0, 1])
def test_grad_hea12(sv, dtype, hea12_reference):
    c, p, obs, e_ref, g_ps, g_fd = hea12_reference
    st = sv.StateVector(12, dtype)
    e, g = st.grad(sv.Plan(c, 9), p, obs)
    assert abs(e - e_ref) <= 1e-6 * max(1.0, abs(e_ref))
    # the target's bar against both references; the complex128 path (FP64 arithmetic
    # and reductions) is also held to 1e-9 of the exact parameter-shift gradient
    assert np.linalg.norm(g - g_ps) <= 1e-4 * np.linalg.norm(g_ps)
    assert np.linalg.norm(g - g_fd) <= 1e-4 * np.linalg.norm(g_fd)
    if dtype == 1:
        assert np.linalg.norm(g - g_ps) <= 1e-9 * np.linalg.norm(g_ps)
    # the backward sweep un-applies the circuit: the state returns to |0...0>
    back = st.get_host().astype(np.complex128)
    assert np.linalg.norm(back - C.zero_state(12)) <= (1e-4 if dtype == 0 else 1e-10)


def test_grad_matches_finite_differences(sv):
    c = C.hea(6, 3)
    p = C.hea_params(c.n_params, 9)
    obs = C.tfim(6)
    st = sv.StateVector(6)
    _, g = st.grad(sv.Plan(c, 4), p, obs)
    g_fd = GR.finite_difference(c, p, obs)
    assert np.linalg.norm(g - g_fd) <= 1e-4 * np.linalg.norm(g_fd)


def test_grad_rx_and_mixed(sv):
    n = 5
    gates = []
    slot = 0
    for layer in range(3):
        for q in range(n):
            gates.append(C.Gate(("RX", "RY", "RZ")[(q + layer) % 3], (q,), slot))
            slot += 1
        for q in range(n - 1):
            gates.append(C.Gate("CZ" if layer % 2 else "CX", (q, q + 1)))
        gates.append(C.Gate("H", (layer % n,)))
        gates.append(C.Gate("SWAP", (0, n - 1)))
    c = C.Circuit(n, gates, slot)
    p = C.hea_params(slot, 1)
    obs = C.Observable(n, C.tfim(n).terms + [(0.3, "XYZIY")])
    st = sv.StateVector(n)
    e, g = st.grad(sv.Plan(c, 3), p, obs)
    assert abs(e - O.expval(S.simulate(c, p), obs)) <= 1e-6 * max(1, abs(e))
    g_ps = GR.parameter_shift(c, p, obs)
    assert np.linalg.norm(g - g_ps) <= 1e-4 * np.linalg.norm(g_ps)


def test_errors_are_reported(sv):
    from paper_2509_14098_gb300 import _native as N
    st = sv.StateVector(5)
    plan = sv.Plan(C.qft(6), 4)
    with pytest.raises(sv.SvError) as e:
        st.run(plan)
    assert e.value.status == N.SV_ERR_ARG
    c = C.Circuit(3, [C.Gate("P", (0,), 0)], n_params=1)
    with pytest.raises(sv.SvError) as e:
        sv.StateVector(3).grad(sv.Plan(c, 2), np.array([0.1]), C.tfim(3))
    assert e.value.status == N.SV_ERR_UNSUPPORTED


def _term_class_observable(n, seed):
    """Pauli terms that reach every path of the sweep planner: diagonal terms on tile
    bits only / global bits only / both, X and Y on the low (lane) bits, the register
    bits, the upper tile bits and mixtures of them, Y with Z on register bits (complex
    coefficients and per-element signs), and X outside the first tile (later sweeps)."""
    def s(**f):
        c = ["I"] * n
        for q, p in f.items():
            c[int(q[1:])] = p
        return "".join(c)
    terms = [(0.9, s(q0="X")), (0.4, s(q1="X", q2="X")), (0.7, s(q5="X")), (0.3, s(q5="X", q13="X")),
             (0.6, s(q5="Y", q7="Z")), (0.5, s(q3="Y", q15="Y")), (0.2, s(q7="X", q9="Y", q11="Z")),
             (0.35, s(q9="X")), (0.25, s(q11="X", q8="Z")), (0.45, s(q13="Y")), (0.15, s(q15="X", q0="Z")),
             (1.0, s(q4="Z", q5="Z")), (0.8, s(q0="Z")), (0.65, s(q1="Z", q9="Z")),
             (0.55, s(q8="Z", q10="Z")), (0.3, s(q12="Z", q14="Z", q10="Z")),
             (0.75, s(q4="Z", q8="Z")), (0.2, s(q5="Z", q12="Z", q7="Z")),
             (0.5, s(q8="X")), (0.4, s(q10="X", q12="Y")), (0.3, s(q14="X", q0="Z")), (0.1, s()),
             ]
    rng = np.random.default_rng(seed)
    for _ in range(20):
        k = int(rng.integers(1, 5))
        qs = rng.choice(n, size=k, replace=False)
        c = ["I"] * n
        for q in qs:
            c[q] = "XYZ"[int(rng.integers(0, 3))]
        terms.append((float(rng.normal()), "".join(c)))
    return C.Observable(n, terms)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("seed", range(3))
def test_expval_term_classes(sv, dtype, seed):
    n = 16
    psi = C.random_state(n, 40 + seed)
    st = sv.StateVector(n, dtype)
    st.set_host(psi)
    obs = _term_class_observable(n, seed)
    e_ref = O.expval(psi, obs)
    tol = 1e-6 * max(1.0, abs(e_ref)) if dtype == 0 else 1e-11 * max(1.0, abs(e_ref))
    assert abs(st.expval(obs) - e_ref) <= tol


def test_grad_term_classes(sv):
    """lambda = O psi over several accumulating sweeps, checked through the gradient."""
    n = 14
    c = C.hea(n, 2)
    p = C.hea_params(c.n_params, 11)
    obs = _term_class_observable(16, 0)
    obs = C.Observable(n, [(cf, ps[:n]) for cf, ps in obs.terms])
    st = sv.StateVector(n)
    e, g = st.grad(sv.Plan(c, 9), p, obs)
    assert abs(e - O.expval(S.simulate(c, p), obs)) <= 1e-6 * max(1.0, abs(e))
    g_ps = GR.parameter_shift(c, p, obs)
    assert np.linalg.norm(g - g_ps) <= 1e-4 * np.linalg.norm(g_ps)


@pytest.mark.parametrize("dtype", [0, 1])
def test_expval_wide_tiles(sv, dtype):
    """21 qubits carrying X: TFIM takes two complex64 sweeps (13 + 8 X qubits: tiles hold
    qubits 0..3 plus up to 9 others after the first) and three complex128 ones (12 + 8 +
    1, the last nearly empty); then a mixed observable on the same state."""
    n = 21
    psi = C.random_state(n, 61)
    st = sv.StateVector(n, dtype)
    st.set_host(psi)
    for obs, sweeps in ((C.tfim(n), 2 if dtype == 0 else 3), (C.Observable(n, C.tfim(n).terms + _term_class_observable(n, 5).terms), None)):
        e_ref = O.expval(psi, obs)
        tol = 1e-6 * max(1.0, abs(e_ref)) if dtype == 0 else 1e-11 * max(1.0, abs(e_ref))
        before = st.run_info()["reduction_sweeps"]
        assert abs(st.expval(obs) - e_ref) <= tol
        if sweeps is not None:
            assert st.run_info()["reduction_sweeps"] - before == sweeps
