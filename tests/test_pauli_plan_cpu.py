"""Host logic of the Pauli-sum sweeps (no GPU): the grouping sv_expval and sv_grad run,
read back through sv_pauli_plan_info.  A sweep's tile holds 13 qubits for complex64 and
12 for complex128 (the whole state below that): qubits 0..3 (128-byte runs) and the X/Y
qubits of its terms; each thread
holds 16 (complex64) or 8 (complex128) elements on register qubits chosen among them.
Every term is evaluated exactly once, the diagonal ones in the first sweep."""
import ctypes
import math

import numpy as np
import pytest

import circuits as C


@pytest.fixture(scope="module")
def N():
    import __graft_entry__ as ge
    ge.build()
    from paper_2509_14098_gb300 import _native as N
    return N


def _plan(N, obs, dtype=0):
    o, keep = N.observable_struct(obs)
    ns = ctypes.c_uint32(0)
    st = N.lib.sv_pauli_plan_info(obs.n_qubits, dtype, ctypes.byref(o), ctypes.byref(ns), None, None, None)
    if st != N.SV_OK:
        return st, None
    k = ns.value
    tm, rm, nt = (ctypes.c_uint64 * k)(), (ctypes.c_uint64 * k)(), (ctypes.c_uint32 * k)()
    N.check(N.lib.sv_pauli_plan_info(obs.n_qubits, dtype, ctypes.byref(o), ctypes.byref(ns), tm, rm, nt))
    return N.SV_OK, (list(tm), list(rm), list(nt))


def _xmask(s):
    return sum(1 << q for q, c in enumerate(s) if c in "XY")


def _tile(dtype):
    return 13 if dtype == 0 else 12


def _check_invariants(obs, plan, dtype):
    tiles, regs, nterms = plan
    n = obs.n_qubits
    T = min(n, _tile(dtype))
    full = (1 << n) - 1
    assert sum(nterms) == len(obs.terms)
    for t, r in zip(tiles, regs):
        assert bin(t).count("1") == T and t & ~full == 0
        if n >= 5:
            assert t & 0xF == 0xF                      # 128-byte runs in every tile
            assert r & 0xF == 0                        # register qubits above the lane runs
        assert r & ~t == 0
        assert bin(r).count("1") == min(4 if dtype == 0 else 3, T - min(4, T - 1))
    n_diag = sum(1 for _, s in obs.terms if _xmask(s) == 0)
    assert nterms[0] >= n_diag
    # every X/Y-carrying term fits the tile of some sweep
    for _, s in obs.terms:
        xm = _xmask(s)
        if xm:
            assert any(xm & ~t == 0 for t in tiles)


@pytest.mark.parametrize("n", [3, 8, 12, 13, 20, 21, 28, 30])
@pytest.mark.parametrize("dtype", [0, 1])
def test_tfim_sweep_count(N, n, dtype):
    obs = C.tfim(n)
    st, plan = _plan(N, obs, dtype)
    assert st == N.SV_OK
    tw = _tile(dtype)
    expect = 1 if n <= tw else 1 + math.ceil((n - tw) / (tw - 4))
    assert len(plan[0]) == expect
    _check_invariants(obs, plan, dtype)
    # the first sweep holds the lowest qubits and every ZZ term
    assert plan[0][0] == (1 << min(n, tw)) - 1
    assert plan[2][0] == (n - 1) + min(n, tw)


@pytest.mark.parametrize("seed", range(6))
def test_random_observables(N, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(13, 33))
    terms = []
    for _ in range(int(rng.integers(20, 80))):
        k = int(rng.integers(1, 7))
        qs = rng.choice(n, size=k, replace=False)
        c = ["I"] * n
        for q in qs:
            c[q] = "IXYZ"[int(rng.integers(0, 4))]
        terms.append((float(rng.normal()), "".join(c)))
    obs = C.Observable(n, terms)
    for dtype in (0, 1):
        st, plan = _plan(N, obs, dtype)
        assert st == N.SV_OK
        _check_invariants(obs, plan, dtype)


def test_register_qubits_follow_the_x_qubits(N):
    # X on qubits 20..27 only, plus the ZZ chain: one sweep whose tile is qubits 0..3, the
    # X qubits and one filler qubit (complex64 tiles hold 13), with the register qubits
    # among the X qubits
    n = 28
    terms = [(1.0, "".join("X" if q == j else "I" for q in range(n))) for j in range(20, 28)]
    terms += C.tfim(n, 0.0).terms[: n - 1]
    obs = C.Observable(n, terms)
    st, plan = _plan(N, obs)
    assert st == N.SV_OK
    tiles, regs, nterms = plan
    xq = sum(1 << j for j in range(20, 28))
    assert tiles == [0xF | xq | 0x10] and nterms == [n - 1 + 8]
    assert regs[0] & ~xq == 0 and bin(regs[0]).count("1") == 4
    # X on 18..29 of 30 qubits (12 X qubits besides 0..3): two sweeps, each X qubit in a tile
    n = 30
    obs = C.Observable(n, [(1.0, "".join("X" if q == j else "I" for q in range(n))) for j in range(18, 30)])
    st, plan = _plan(N, obs)
    assert st == N.SV_OK and len(plan[0]) == 2
    _check_invariants(obs, plan, 0)


@pytest.mark.parametrize("dtype", [0, 1])
def test_term_too_wide_is_rejected(N, dtype):
    n, tw = 20, _tile(dtype)
    fits = "".join("X" if 4 <= q < tw else "I" for q in range(n))      # tw - 4 X outside qubits 0..3
    wide = "".join("X" if 4 <= q < tw + 1 else "I" for q in range(n))  # one more
    st, plan = _plan(N, C.Observable(n, [(1.0, fits)]), dtype)
    assert st == N.SV_OK and len(plan[0]) == 1
    st, _ = _plan(N, C.Observable(n, [(1.0, wide)]), dtype)
    assert st == N.SV_ERR_UNSUPPORTED
    # qubits 0..3 count toward the tile: 4 + (tw - 4) fit
    st, _ = _plan(N, C.Observable(n, [(1.0, "".join("X" if q < tw else "I" for q in range(n)))]), dtype)
    assert st == N.SV_OK


def test_bad_arguments(N):
    obs = C.tfim(8)
    o, keep = N.observable_struct(obs)
    ns = ctypes.c_uint32(0)
    assert N.lib.sv_pauli_plan_info(9, 0, ctypes.byref(o), ctypes.byref(ns), None, None, None) == N.SV_ERR_ARG
    assert N.lib.sv_pauli_plan_info(8, 7, ctypes.byref(o), ctypes.byref(ns), None, None, None) == N.SV_ERR_ARG
    tm = (ctypes.c_uint64 * 1)()
    ns.value = 0
    assert N.lib.sv_pauli_plan_info(8, 0, ctypes.byref(o), ctypes.byref(ns), tm, None, None) == N.SV_ERR_ARG
