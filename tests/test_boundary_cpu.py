"""Host-side boundary tests (no GPU): the library loads, exports every entry point
include/sv.h declares, and its C++ partitioner reproduces the oracle's partition
exactly (stage local sets, gate order, final map, closeness integers)."""
import os
import re
import subprocess

import numpy as np
import pytest

import circuits as C
from oracle import partition as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def sv():
    import __graft_entry__ as ge
    ge.build()
    import paper_2509_14098_gb300 as pkg
    return pkg


def _declared():
    txt = open(os.path.join(ROOT, "include", "sv.h")).read()
    return sorted(set(re.findall(r"^\s*(?:sv_status|const char\*)\s+(sv_\w+)\s*\(", txt, re.M)))


def test_exports_every_declared_symbol(sv):
    from paper_2509_14098_gb300 import _native as N
    out = subprocess.run(["nm", "-D", "--defined-only", N.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (sv_\w+)", out))
    declared = _declared()
    assert declared, "no declarations parsed"
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    for s in declared:
        assert hasattr(N.lib, s)


def _oracle_partition(c, L, nf):
    stages, final = P.partition(c, L, range(min(nf, L, c.n_qubits)))
    return [(sum(1 << b for b in loc), ids) for loc, ids in stages], final


def _native_partition(sv, c, L, nf):
    plan = sv.Plan(c, L, nf)
    st = plan.stages()
    order, fmap = plan.order()
    out, k = [], 0
    for mask, cnt in st:
        out.append((mask, order[k:k + cnt]))
        k += cnt
    return out, fmap, plan


CASES = [(C.ghz(3), 2, 0), (C.ghz(9), 3, 0), (C.qft(8), 3, 0), (C.qft(10), 5, 4),
         (C.brickwork(10, 6, 1), 4, 2), (C.hea(7, 3), 6, 4), (C.qft_roundtrip(12), 6, 4),
         (C.Circuit(5, []), 3, 0)]   # the empty circuit: no stages


@pytest.mark.parametrize("c,L,nf", CASES)
def test_partition_bit_exact(sv, c, L, nf):
    ref, ref_final = _oracle_partition(c, L, nf)
    got, got_final, plan = _native_partition(sv, c, L, nf)
    assert got == ref
    assert got_final == ref_final
    cc, size, dist, level = P.closeness(c)
    r, d, lv = plan.centrality()
    assert r == size and d == dist and lv == level


def test_partition_closeness_choice_golden(sv):
    """The C++ partitioner on the hand-derived closeness-choice cases (Sec. 4.2)."""
    import json
    cases = json.load(open(os.path.join(ROOT, "tests", "golden", "cc_choice.json")))["cases"]
    for case in cases:
        c = C.Circuit(case["n_qubits"], [C.Gate(k, tuple(q)) for k, q in case["gates"]])
        got, _, plan = _native_partition(sv, c, case["L"], 0)
        want = [(sum(1 << b for b in s["local"]), s["gates"]) for s in case["stages"]]
        assert got == want, case["name"]
        r, d, lv = plan.centrality()
        assert r == [len(x) for x in case["reach"]] and d == case["dist"] and lv == case["levels"]


@pytest.mark.parametrize("seed", range(12))
def test_partition_bit_exact_random(sv, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 9))
    c = C.random_circuit(n, int(rng.integers(5, 80)), seed)
    L = int(rng.integers(1, n + 1))
    nf = int(rng.integers(0, 3))
    try:
        ref = _oracle_partition(c, L, nf)
    except P.PartitionError:
        with pytest.raises(sv.SvError) as e:
            sv.Plan(c, L, nf)
        assert e.value.status == 4
        return
    got = _native_partition(sv, c, L, nf)
    assert got[0] == ref[0] and got[1] == ref[1]


@pytest.mark.parametrize("name", ["brick16", "qft30", "brick32", "hea28"])
def test_config_partitions_bit_exact(sv, name):
    c, _, L = C.workload(name)
    ref = _oracle_partition(c, L, 4)
    got = _native_partition(sv, c, L, 4)
    assert got[0] == ref[0] and got[1] == ref[1]


def test_partition_errors(sv):
    from paper_2509_14098_gb300 import _native as N
    with pytest.raises(sv.SvError) as e:
        sv.Plan(C.ghz(4), 0)
    assert e.value.status == N.SV_ERR_ARG
    bad = C.Circuit(3, [C.Gate("H", (0,))])
    object.__setattr__(bad.gates[0], "qubits", (5,))
    with pytest.raises(sv.SvError) as e:
        sv.Plan(bad, 2)
    assert e.value.status == N.SV_ERR_ARG
    c = C.Circuit(2, [C.Gate("RY", (0,), 3)], n_params=2)
    with pytest.raises(sv.SvError):
        sv.Plan(c, 2)


def test_state_calls_fail_loudly_without_gpu(sv):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import ctypes
    from paper_2509_14098_gb300 import _native as N
    h = ctypes.c_void_p()
    st = N.lib.sv_create(4, 0, None, None, ctypes.byref(h))
    assert st == N.SV_ERR_CUDA
