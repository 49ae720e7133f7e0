"""Host planning of the permutation sweep (the on-GPU form of the inter-partition data
reshaping, Sec. 4.3), checked on the CPU through sv_permute_plan_info: the tile holds the
input's 4 lowest bits and the input bits of output bits 0..3, has the dtype's width, and
its contiguous input and output runs are both at least 512 bytes, so both the reads and
the writes of the sweep are long coalesced runs (the data movement itself is checked
bit-exact on the GPU in test_gpu_parity.py)."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def sv():
    import __graft_entry__ as ge
    ge.build()
    import paper_2509_14098_gb300 as pkg
    return pkg


def plan(sv, n, dtype, perm):
    from paper_2509_14098_gb300 import _native as N
    arr = (ctypes.c_uint32 * n)(*perm)
    T, ri, ro = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    mask = ctypes.c_uint64()
    N.check(N.lib.sv_permute_plan_info(n, dtype, arr, ctypes.byref(T), ctypes.byref(mask), ctypes.byref(ri),
                                       ctypes.byref(ro)))
    return T.value, mask.value, ri.value, ro.value


def check(n, dtype, perm, T, mask, ri, ro):
    eb = 8 if dtype == 0 else 16
    assert T == min(n, 12 if dtype == 0 else 11)
    assert bin(mask).count("1") == T and mask < (1 << n)
    for b in range(min(4, n)):
        assert (mask >> b) & 1                 # the input's lowest bits
        assert (mask >> perm[b]) & 1           # the input bit that becomes output bit b
    # the runs the sweep relies on, recomputed from the mask
    r_in = 0
    while r_in < n and (mask >> r_in) & 1:
        r_in += 1
    r_out = 0
    while r_out < n and (mask >> perm[r_out]) & 1:
        r_out += 1
    assert (ri, ro) == (r_in, r_out)
    if n >= T + 1:
        assert (eb << ri) >= 512 and (eb << ro) >= 512, (ri, ro)


@pytest.mark.parametrize("dtype", [0, 1])
def test_bit_reversal(sv, dtype):
    n = 30
    perm = list(range(n))[::-1]
    T, mask, ri, ro = plan(sv, n, dtype, perm)
    check(n, dtype, perm, T, mask, ri, ro)
    assert mask & 0xF == 0xF and (mask >> 26) & 0xF == 0xF


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("seed", range(20))
def test_random_permutations(sv, dtype, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 37))
    perm = [int(x) for x in rng.permutation(n)]
    check(n, dtype, perm, *plan(sv, n, dtype, perm))


def test_rejects_non_permutations(sv):
    with pytest.raises(sv.SvError) as e:
        plan(sv, 5, 0, [0, 1, 1, 3, 4])
    assert e.value.status == 1
    with pytest.raises(sv.SvError):
        plan(sv, 5, 0, [0, 1, 2, 3, 5])
