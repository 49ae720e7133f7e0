"""Host logic of the tensor-core stages (no GPU), read back through sv_gemm_plan_info:
B residency and ring depth per fusion width, and the producer lane mapping.  The
operand layout is the 128-byte-swizzled K-major one (rows of 128 bytes, 8-row groups
of 1 KB, the 16-byte unit index XORed with the row index within its group); a K chunk
row holds 16 TF32 (re, im) amplitudes (8 bytes each) or 32 BF16 ones (4 bytes).  A
warp's operand stores are free of shared-memory bank conflicts when the lanes that
share a wavefront (128 bytes per wavefront) write distinct 4-byte-bank groups."""
import ctypes

import pytest

import circuits as C


@pytest.fixture(scope="module")
def N():
    import __graft_entry__ as ge
    ge.build()
    from paper_2509_14098_gb300 import _native as N
    return N


def _info(N, circ, k, prec):
    plan = ctypes.c_void_p()
    c, keep = N.circuit_struct(circ)
    N.check(N.lib.sv_partition_gemm(ctypes.byref(c), k, ctypes.byref(plan)))
    try:
        ns = ctypes.c_uint32(0)
        N.check(N.lib.sv_gemm_plan_info(plan, None, prec, ctypes.byref(ns), None, None, None, None))
        m = ns.value
        keff, res, nslot = (ctypes.c_uint32 * m)(), (ctypes.c_uint32 * m)(), (ctypes.c_uint32 * m)()
        roles = (ctypes.c_uint8 * (6 * m))()
        N.check(N.lib.sv_gemm_plan_info(plan, None, prec, ctypes.byref(ns), keff, res, nslot, roles))
        return list(keff), list(res), list(nslot), [list(roles[6 * s:6 * s + 6]) for s in range(m)]
    finally:
        N.lib.sv_plan_destroy(plan)


def _offset(prec, jj, m):
    """Byte offset of amplitude jj of operand row m in the swizzled layout."""
    b = jj * (8 if prec == 1 else 4)                 # byte inside the 128-byte row
    return (m // 8) * 1024 + (m % 8) * 128 + (((b // 16) ^ (m % 8)) * 16) + b % 16


def _lanes_conflict_free(prec, roles):
    pair = roles[5]
    g = (8 if prec == 1 else 4) * (2 if pair == 0 else 1)   # bytes per store
    phase = min(32, 128 // g)                               # lanes per wavefront
    nbits = phase.bit_length() - 1
    slots = set()
    for lane in range(phase):
        jj = m = 0
        active = True
        for i in range(nbits):
            if (lane >> i) & 1:
                r = roles[i]
                if r == 255:
                    active = False
                elif r < 8:
                    jj |= 1 << r
                else:
                    m |= 1 << (r - 8)
        if not active:
            continue
        off = _offset(prec, jj, m)
        slot = (off % 128) // g
        if slot in slots:
            return False
        slots.add(slot)
    return True


@pytest.mark.parametrize("n", [10, 13, 16, 20, 26, 32])
@pytest.mark.parametrize("k", [5, 6, 7])
@pytest.mark.parametrize("prec", [1, 2])
def test_stage_layout(N, n, k, prec):
    if n < k + 4:
        pytest.skip("narrower than the stage needs")
    circ = C.brickwork(n, 8, 3)
    keff, res, nslot, roles = _info(N, circ, k, prec)
    assert keff and all(e == max(6, k) for e in keff)
    for e, r, ns, ro in zip(keff, res, nslot, roles):
        assert r == (1 if e == 6 else 0)                   # B stays resident up to 6 local qubits
        assert ns in (2, 3)
        # the pair bit is the lowest chunk-varying bit: amplitude bit 0 or column bit 0
        assert ro[5] in (0, 8)
        # lane bits select distinct chunk-varying bits
        sel = [x for x in ro[:5] if x != 255]
        assert len(set(sel)) == len(sel) and ro[5] not in sel
        assert _lanes_conflict_free(prec, ro), (n, k, prec, ro)


def test_lowest_bits_mapping_would_conflict(N):
    """The check above has teeth: with local qubits above the column bits (pair bit =
    column bit 0) the plain lowest-bits lane choice (column bits 1..5) puts 8 lanes on
    one bank group."""
    assert not _lanes_conflict_free(2, [9, 10, 11, 12, 13, 8])
    assert _lanes_conflict_free(2, [9, 10, 0, 1, 2, 8])


def test_not_a_tensor_core_plan(N):
    circ = C.brickwork(12, 2, 1)
    plan = ctypes.c_void_p()
    c, keep = N.circuit_struct(circ)
    N.check(N.lib.sv_partition(ctypes.byref(c), 8, ctypes.byref(plan)))
    ns = ctypes.c_uint32(0)
    try:
        assert N.lib.sv_gemm_plan_info(plan, None, 2, ctypes.byref(ns), None, None, None, None) == N.SV_ERR_UNSUPPORTED
        assert N.lib.sv_gemm_plan_info(plan, None, 0, ctypes.byref(ns), None, None, None, None) == N.SV_ERR_ARG
    finally:
        N.lib.sv_plan_destroy(plan)


def test_hierarchical_plan_shape(N):
    """sv_partition_hier: level-1 stages of k + 7 qubits holding 0..3; level 2 packs a
    stage's gates into k-qubit sub-partitions, so brick32 needs far fewer HBM passes
    than the flat tensor-core plan (one pass per fused unitary)."""
    import paper_2509_14098_gb300 as sv
    circ = C.brickwork(32, 24, 3)
    for k in (5, 6):
        plan = sv.Plan(circ, k, hier=True)
        st = plan.stages()
        assert all(bin(m).count("1") == k + 7 and m & 15 == 15 for m, _ in st)
        nl, ns = plan.hier_info(2)
        flat = sv.Plan(circ, k, gemm=True)
        assert nl == len(st) < len(flat.stages()) <= ns
    nl, ns = sv.Plan(circ, 5, hier=True).hier_info(1)
    assert ns > nl > 0


def test_hierarchical_plan_errors(N):
    import paper_2509_14098_gb300 as sv
    with pytest.raises(N.SvError):
        sv.Plan(C.brickwork(16, 2, 1), 7, hier=True)      # k must be 5 or 6
    with pytest.raises(N.SvError):
        sv.Plan(C.brickwork(11, 2, 1), 5, hier=True)      # narrower than one tile
    plan = sv.Plan(C.brickwork(14, 2, 1), 6, hier=True)
    with pytest.raises(N.SvError):
        plan.hier_info(1)                                 # TF32x3 needs k = 5
    with pytest.raises(N.SvError):
        sv.Plan(C.brickwork(14, 2, 1), 8).hier_info(2)    # not a hierarchical plan


def test_hierarchical_long_stage_takes_several_launches(N):
    """A stage with more than 24 sub-partitions is split into launches of at most 24."""
    import paper_2509_14098_gb300 as sv
    circ = C.Circuit(14, C.random_circuit(12, 700, 3).gates)
    plan = sv.Plan(circ, 5, hier=True)
    nl, ns = plan.hier_info(2)
    assert len(plan.stages()) == 1 and ns > 24 and nl == (ns + 23) // 24
