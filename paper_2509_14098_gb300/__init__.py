"""GB300-native execution of closeness-centrality-partitioned quantum circuits.

Python surface over the C ABI (include/sv.h): partition a circuit on the host
(Plan), then run it on a state vector held in GPU memory (StateVector).  PyTorch
provides device memory and streams only; every state operation runs in this
package's CUDA kernels.
"""
import ctypes

import numpy as np

from . import _native as N
from ._native import SvError, SV_C64, SV_C128, SV_PREC_CUDACORE, SV_PREC_TF32X3, SV_PREC_BF16X3, SV_PREC_NO_RENORM

__all__ = ["Plan", "StateVector", "Batch", "SvError", "partition", "parse_qasm", "SV_C64", "SV_C128",
           "SV_PREC_CUDACORE", "SV_PREC_TF32X3", "SV_PREC_BF16X3", "SV_PREC_NO_RENORM"]

_KIND_NAMES = {v: k for k, v in N.GATE_CODES.items()}
_N_ANGLES = {"RX": 1, "RY": 1, "RZ": 1, "P": 1, "CP": 1, "U3": 3}


class QasmGate:
    """One gate of a parsed circuit: kind name, qubits (control first), fixed angles."""
    __slots__ = ("kind", "qubits", "param", "angles")

    def __init__(self, kind, qubits, angles):
        self.kind, self.qubits, self.param, self.angles = kind, tuple(qubits), -1, tuple(angles)

    def __repr__(self):
        return f"QasmGate({self.kind}, {self.qubits}, {self.angles})"


class QasmCircuit:
    """A flat gate list read from OpenQASM 2.0 text (sv_qasm_parse); Plan accepts it."""

    def __init__(self, n_qubits, gates):
        self.n_qubits, self.gates, self.n_params, self.name = n_qubits, gates, 0, "qasm"


def parse_qasm(text):
    """Parse OpenQASM 2.0 text (the subset sv_qasm_parse documents) into a QasmCircuit."""
    src = text.encode() if isinstance(text, str) else bytes(text)
    nq, ng = ctypes.c_uint32(), ctypes.c_uint32()
    N.check(N.lib.sv_qasm_parse(src, None, 0, ctypes.byref(nq), ctypes.byref(ng)))
    arr = (N.sv_gate * max(1, ng.value))()
    N.check(N.lib.sv_qasm_parse(src, arr, ng.value, ctypes.byref(nq), ctypes.byref(ng)))
    gates = []
    for i in range(ng.value):
        g = arr[i]
        kind = _KIND_NAMES[g.kind]
        gates.append(QasmGate(kind, [g.q[k] for k in range(g.nq)], [g.angle[k] for k in range(_N_ANGLES.get(kind, 0))]))
    return QasmCircuit(nq.value, gates)


class Plan:
    """Host-side partition of a circuit (sv_partition / sv_partition_ex)."""

    def __init__(self, circuit, L, n_fixed=None, gemm=False, hier=False):
        """gemm=True: partition for tensor-core stages (sv_partition_gemm, L = fusion width k);
        hier=True: hierarchical tensor-core stages (sv_partition_hier, L = sub-partition
        width k, tiles of k + 7 qubits)."""
        self.circuit = circuit
        self.L = L
        c, self._gates = N.circuit_struct(circuit)
        self._c = c
        h = ctypes.c_void_p()
        if hier:
            N.check(N.lib.sv_partition_hier(ctypes.byref(c), L, ctypes.byref(h)))
        elif gemm:
            N.check(N.lib.sv_partition_gemm(ctypes.byref(c), L, ctypes.byref(h)))
        elif n_fixed is None:
            N.check(N.lib.sv_partition(ctypes.byref(c), L, ctypes.byref(h)))
        else:
            N.check(N.lib.sv_partition_ex(ctypes.byref(c), L, n_fixed, ctypes.byref(h)))
        self.handle = h

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            N.lib.sv_plan_destroy(h)
            self.handle = None

    def hier_info(self, prec, params=None):
        """(stage launches, sub-partitions in all) of a hierarchical plan (sv_hier_plan_info)."""
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
        nl, ns = ctypes.c_uint32(), ctypes.c_uint32()
        N.check(N.lib.sv_hier_plan_info(self.handle, N.as_double_ptr(p), prec, ctypes.byref(nl), ctypes.byref(ns)))
        return nl.value, ns.value

    def stages(self):
        """[(local physical-bit mask, gate count)] per stage."""
        n = ctypes.c_uint32(0)
        N.check(N.lib.sv_plan_stages(self.handle, ctypes.byref(n), None, None))
        masks = (ctypes.c_uint64 * n.value)()
        counts = (ctypes.c_uint32 * n.value)()
        N.check(N.lib.sv_plan_stages(self.handle, ctypes.byref(n), masks, counts))
        return [(int(masks[i]), int(counts[i])) for i in range(n.value)]

    def order(self):
        """(gate ids in execution order, final map circuit qubit -> physical bit)."""
        G, n = len(self.circuit.gates), self.circuit.n_qubits
        order = (ctypes.c_uint32 * G)()
        fmap = (ctypes.c_uint32 * n)()
        N.check(N.lib.sv_plan_order(self.handle, order, fmap))
        return list(order), list(fmap)

    def compile(self, params=None, forward=True, adjoint=False):
        """Generate and compile the plan's complex64 stage kernels ahead of the first
        run (sv_plan_compile); returns the number of stage kernels."""
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
        which = (1 if forward else 0) | (2 if adjoint else 0)
        n = ctypes.c_uint32(0)
        N.check(N.lib.sv_plan_compile(self.handle, N.as_double_ptr(p), which, ctypes.byref(n)))
        return n.value

    def centrality(self):
        """(|RN|, dist, level) per gate."""
        G = len(self.circuit.gates)
        r = (ctypes.c_uint32 * G)()
        d = (ctypes.c_uint64 * G)()
        lv = (ctypes.c_uint32 * G)()
        N.check(N.lib.sv_plan_centrality(self.handle, r, d, lv))
        return list(r), list(d), list(lv)


def partition(circuit, L, n_fixed=None):
    return Plan(circuit, L, n_fixed)


class StateVector:
    """A state of n qubits in GPU memory (a borrowed torch tensor of complex64 /
    complex128), bound to a CUDA stream."""

    def __init__(self, n_qubits, dtype=SV_C64, tensor=None, device="cuda", stream=None):
        import torch
        self.n = n_qubits
        self.dtype = dtype
        tdt = torch.complex64 if dtype == SV_C64 else torch.complex128
        if tensor is None:
            tensor = torch.zeros(1 << n_qubits, dtype=tdt, device=device)
            tensor[0] = 1
        if tensor.dtype != tdt or tensor.numel() != (1 << n_qubits) or not tensor.is_cuda or not tensor.is_contiguous():
            raise ValueError("state tensor must be a contiguous CUDA tensor of 2^n amplitudes of the dtype")
        self.tensor = tensor
        self.stream = stream if stream is not None else torch.cuda.current_stream(tensor.device)
        h = ctypes.c_void_p()
        N.check(N.lib.sv_create(n_qubits, dtype, ctypes.c_void_p(tensor.data_ptr()),
                                ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.handle = h

    def close(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            N.lib.sv_destroy(h)
            self.handle = None

    def __del__(self):
        self.close()

    # --- state movement -------------------------------------------------------
    def reset(self):
        N.check(N.lib.sv_reset_zero(self.handle))

    def set_host(self, array):
        a = np.ascontiguousarray(array, dtype=np.complex64 if self.dtype == SV_C64 else np.complex128)
        N.check(N.lib.sv_set_state_host(self.handle, a.ctypes.data_as(ctypes.c_void_p)))
        self.synchronize()   # the host array may be pageable and temporary

    def get_host(self):
        out = np.empty(1 << self.n, dtype=np.complex64 if self.dtype == SV_C64 else np.complex128)
        N.check(N.lib.sv_get_state_host(self.handle, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def synchronize(self):
        N.check(N.lib.sv_synchronize(self.handle))

    # --- execution ------------------------------------------------------------
    def run(self, plan, params=None, prec=SV_PREC_CUDACORE):
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
        self._params = p
        N.check(N.lib.sv_run(self.handle, plan.handle, N.as_double_ptr(p), prec))

    def permute(self, phys_of_qubit):
        arr = (ctypes.c_uint32 * self.n)(*phys_of_qubit)
        N.check(N.lib.sv_permute(self.handle, arr))

    def norm(self):
        out = ctypes.c_double()
        N.check(N.lib.sv_norm(self.handle, ctypes.byref(out)))
        return out.value

    def expval(self, obs):
        o, keep = N.observable_struct(obs)
        out = ctypes.c_double()
        N.check(N.lib.sv_expval(self.handle, ctypes.byref(o), ctypes.byref(out)))
        return out.value

    def grad(self, plan, params, obs):
        """Adjoint gradient; returns (E, dE/dtheta).  The state after the call is the
        backward pass's reconstruction of the input state."""
        p = np.ascontiguousarray(params, dtype=np.float64)
        o, keep = N.observable_struct(obs)
        e = ctypes.c_double()
        g = np.zeros(max(1, len(p)), dtype=np.float64)
        N.check(N.lib.sv_grad(self.handle, plan.handle, N.as_double_ptr(p), ctypes.byref(o),
                              ctypes.byref(e), N.as_double_ptr(g)))
        return e.value, g[: len(p)]

    def timing(self, enable=None, reset=False):
        """Enable / disable per-kernel event timing, or read the accumulated record."""
        if enable is not None:
            N.check(N.lib.sv_timing_enable(self.handle, 1 if enable else 0))
            return None
        t = N.sv_timing()
        N.check(N.lib.sv_timing_read(self.handle, ctypes.byref(t), 1 if reset else 0))
        return {f: getattr(t, f) for f, _ in N.sv_timing._fields_}

    def run_info(self):
        info = N.sv_run_info()
        N.check(N.lib.sv_last_run_info(self.handle, ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in N.sv_run_info._fields_}


class Batch:
    """Many circuits evaluated together (sv_batch_create / sv_run_batch): E_i =
    <psi_i|O_i|psi_i> and dE_i/dtheta for every circuit, in one persistent launch
    replayed from a captured CUDA graph.  observables: one Z-string sum per circuit.
    tune: {n: (L, k)} or None."""

    def __init__(self, circuits, observables, tune=None, stream=None):
        if len(circuits) != len(observables):
            raise ValueError("one observable per circuit")
        self.n_params = [c.n_params for c in circuits]
        self.total_params = sum(self.n_params)
        cs = (N.sv_circuit * len(circuits))()
        os_ = (N.sv_observable * len(circuits))()
        keep = []
        for i, (c, o) in enumerate(zip(circuits, observables)):
            cst, arr = N.circuit_struct(c)
            ost, ok = N.observable_struct(o)
            cs[i] = cst
            os_[i] = ost
            keep.append((arr, ok))
        t = None
        if tune:
            t = N.sv_tune()
            for n, (L, k) in tune.items():
                t.L[n], t.k[n] = L, k
        h = ctypes.c_void_p()
        st = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        N.check(N.lib.sv_batch_create(cs, os_, len(circuits), None if t is None else ctypes.byref(t), st,
                                      ctypes.byref(h)))
        self.n = len(circuits)
        self.handle = h

    def close(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            N.lib.sv_batch_destroy(h)
            self.handle = None

    def __del__(self):
        self.close()

    def _params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float64).reshape(-1)
        if p.size != self.total_params:
            raise ValueError(f"expected {self.total_params} parameters, got {p.size}")
        return p

    def run(self, params):
        """(E per circuit, gradient in the parameters' layout)."""
        p = self._params(params)
        e = np.zeros(self.n, dtype=np.float64)
        g = np.zeros(max(1, self.total_params), dtype=np.float64)
        N.check(N.lib.sv_run_batch(self.handle, N.as_double_ptr(p), N.as_double_ptr(e), N.as_double_ptr(g)))
        return e, g[: self.total_params]

    def autotune(self, params):
        """Time (L, k) candidates per width, rebuild with the best; returns {n: (L, k)}."""
        p = self._params(params)
        t = N.sv_tune()
        N.check(N.lib.sv_autotune(self.handle, N.as_double_ptr(p), ctypes.byref(t)))
        return {n: (t.L[n], t.k[n]) for n in range(41) if t.L[n]}

    def info(self):
        i = N.sv_batch_info()
        N.check(N.lib.sv_batch_info_get(self.handle, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in N.sv_batch_info._fields_ if f != "pad"}
