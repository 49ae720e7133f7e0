"""Host-side checks of the generated stage kernels (no GPU): for plans of every gate
kind, the generator emits one kernel per stage and direction and NVRTC compiles them
for sm_103a (sv_plan_compile); kernels are cached by source, so a plan of the same
structure with other angle values reuses them.  Their numerics are the GPU parity
tests' subject (tests/test_gpu_*.py run every sv_run / sv_grad on these kernels)."""
import numpy as np
import pytest

import circuits as C


@pytest.fixture(scope="module")
def sv():
    import __graft_entry__ as ge
    ge.build()
    import paper_2509_14098_gb300 as pkg
    return pkg


CASES = [
    ("qft12", lambda: (C.qft_roundtrip(12), None, 6), False),
    ("brick12", lambda: (C.brickwork(12, 6, 1), None, 8), False),
    ("hea10", lambda: (C.hea(10, 3), C.hea_params(60, 1), 7), True),
    ("random", lambda: (C.random_circuit(9, 120, 4), None, 6), False),
    ("ghz14", lambda: (C.ghz(14), None, 5), False),
]


@pytest.mark.parametrize("name,make,adjoint", CASES, ids=[c[0] for c in CASES])
def test_generated_kernels_compile(sv, name, make, adjoint):
    c, p, L = make()
    plan = sv.Plan(c, L)
    n_stages = len(plan.stages())
    assert plan.compile(p, forward=True) == n_stages
    if adjoint:
        assert plan.compile(p, forward=False, adjoint=True) == n_stages
        assert plan.compile(p, forward=True, adjoint=True) == 2 * n_stages


def test_generated_kernels_are_reused_across_angles(sv):
    from paper_2509_14098_gb300 import _native as N
    import ctypes
    c = C.hea(8, 2)
    plan = sv.Plan(c, 6)
    plan.compile(C.hea_params(c.n_params, 1), adjoint=True)
    # the same structure with other angles: only cache hits (the kernel source holds
    # no angle values)
    before = _compiles(N)
    plan.compile(C.hea_params(c.n_params, 2), adjoint=True)
    assert _compiles(N) == before


def _compiles(N):
    import ctypes
    n = ctypes.c_uint64()
    N.check(N.lib.sv_jit_stats(ctypes.byref(n), None, None))
    return n.value


def test_compile_errors(sv):
    from paper_2509_14098_gb300 import _native as N
    c = C.brickwork(10, 2, 1)
    with pytest.raises(sv.SvError) as e:
        sv.Plan(c, 6, gemm=True).compile()
    assert e.value.status == N.SV_ERR_UNSUPPORTED
    h = C.hea(6, 1)
    with pytest.raises(sv.SvError) as e:
        sv.Plan(h, 4).compile(None)                  # parametric circuit without params
    assert e.value.status == N.SV_ERR_ARG


def test_pauli_expectation_kernels_compile(sv):
    """The expectation-only Pauli sweeps (one generated kernel per sweep, terms compiled
    in) are generated and NVRTC-compiled for sm_103a on the host; complex128 keeps the
    generic sweep kernel; a second call is served from the cache."""
    import ctypes
    from paper_2509_14098_gb300 import _native as N
    for n, sweeps in ((12, 1), (20, 2), (30, 3)):
        o, keep = N.observable_struct(C.tfim(n))
        k = ctypes.c_uint32(99)
        N.check(N.lib.sv_pauli_compile(n, 0, ctypes.byref(o), ctypes.byref(k)))
        assert k.value == sweeps
        N.check(N.lib.sv_pauli_compile(n, 1, ctypes.byref(o), ctypes.byref(k)))
        assert k.value == 0
    obs = C.Observable(16, C.tfim(16).terms + [(0.3, "XYZ" + "I" * 10 + "ZYX")])
    o, keep = N.observable_struct(obs)
    k = ctypes.c_uint32(0)
    N.check(N.lib.sv_pauli_compile(16, 0, ctypes.byref(o), ctypes.byref(k)))
    before = _compiles(N)
    N.check(N.lib.sv_pauli_compile(16, 0, ctypes.byref(o), ctypes.byref(k)))
    assert k.value >= 1 and _compiles(N) == before
