"""sv_norm_noalloc: the norm reduction for callers that cannot allocate device memory
(their memory belongs to their own allocator, or an allocation's implicit device
synchronisation is not acceptable where they call).  Its partial sums live in a static
device array; it must agree with the oracle's ||psi||^2 (complex128, on the host copy of
the same state) and with sv_norm, the allocating entry point, on consecutive calls (the
shared array keeps the previous call's contents)."""
import ctypes

import numpy as np
import pytest

from oracle import observables as O

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


def _state(n, dtype, seed, scale):
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    tdt = torch.complex64 if dtype == 0 else torch.complex128
    return torch.randn(1 << n, dtype=tdt, device="cuda", generator=g) * scale


@pytest.mark.parametrize("dtype", [0, 1])
def test_noalloc_norm_matches_sv_norm(sv, dtype):
    import torch
    from paper_2509_14098_gb300 import _native as N
    tol = 1e-6 if dtype == 0 else 1e-12
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row: a larger state first, then a smaller one (fewer partials)
    for n, seed, scale in ((21, 1, 0.01), (13, 2, 0.3)):
        psi = _state(n, dtype, seed, scale)
        st = sv.StateVector(n, dtype, tensor=psi)
        ref = st.norm()
        oref = O.norm2(psi.cpu().numpy().astype(np.complex128))
        N.check(N.lib.sv_norm_noalloc(ctypes.c_void_p(psi.data_ptr()), n, dtype, ctypes.c_void_p(stream),
                                      ctypes.c_void_p(out.data_ptr())))
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= tol * max(1.0, abs(ref)), (n, got, ref)
        assert abs(got - oref) <= tol * max(1.0, abs(oref)), (n, got, oref)
        st.close()


def test_noalloc_rejects_oversize(sv):
    import torch
    from paper_2509_14098_gb300 import _native as N
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    psi = torch.zeros(16, dtype=torch.complex64, device="cuda")
    st = N.lib.sv_norm_noalloc(ctypes.c_void_p(psi.data_ptr()), 33, 0, None, ctypes.c_void_p(out.data_ptr()))
    assert st == N.SV_ERR_ARG
    assert b"32" in N.lib.sv_last_error()
