"""ctypes binding of the C ABI in include/sv.h (argument marshalling only).

Every state operation runs in the library's CUDA kernels; there is no CPU
fallback.  If the shared library is missing, importing this module raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsvgb300.so")

SV_OK, SV_ERR_ARG, SV_ERR_OOM, SV_ERR_CUDA, SV_ERR_PARTITION, SV_ERR_UNSUPPORTED, SV_ERR_TIMEOUT = range(7)
SV_C64, SV_C128 = 0, 1
SV_PREC_CUDACORE, SV_PREC_TF32X3, SV_PREC_BF16X3 = 0, 1, 2
SV_PREC_NO_RENORM = 0x100   # OR-ed into a tensor-core mode: keep the raw split-precision result
STATUS_NAMES = {0: "SV_OK", 1: "SV_ERR_ARG", 2: "SV_ERR_OOM", 3: "SV_ERR_CUDA", 4: "SV_ERR_PARTITION",
                5: "SV_ERR_UNSUPPORTED", 6: "SV_ERR_TIMEOUT"}

GATE_CODES = {k: i + 1 for i, k in enumerate(
    ("H", "X", "Y", "Z", "S", "SDG", "T", "TDG", "RX", "RY", "RZ", "P", "U3", "CX", "CY", "CZ", "CP", "SWAP"))}
PAULI_CODES = {"I": 0, "X": 1, "Y": 2, "Z": 3}


class SvError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class sv_gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint16), ("nq", ctypes.c_uint8), ("q", ctypes.c_uint8 * 3),
                ("reserved", ctypes.c_uint16), ("param", ctypes.c_int32), ("angle", ctypes.c_double * 3)]


class sv_circuit(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_uint32), ("n_gates", ctypes.c_uint32), ("n_params", ctypes.c_uint32),
                ("gates", ctypes.POINTER(sv_gate))]


class sv_observable(ctypes.Structure):
    _fields_ = [("n_terms", ctypes.c_uint32), ("n_qubits", ctypes.c_uint32),
                ("pauli", ctypes.POINTER(ctypes.c_uint8)), ("coeff", ctypes.POINTER(ctypes.c_double))]


class sv_run_info(ctypes.Structure):
    _fields_ = [("stage_sweeps", ctypes.c_uint32), ("permutation_sweeps", ctypes.c_uint32),
                ("reduction_sweeps", ctypes.c_uint32), ("backward_sweeps", ctypes.c_uint32),
                ("kernel_launches", ctypes.c_uint32), ("hbm_bytes", ctypes.c_double)]


class sv_timing(ctypes.Structure):
    _fields_ = [("stage_ms", ctypes.c_double), ("backward_ms", ctypes.c_double), ("permute_ms", ctypes.c_double),
                ("observable_ms", ctypes.c_double), ("stage_launches", ctypes.c_uint32),
                ("backward_launches", ctypes.c_uint32), ("permute_launches", ctypes.c_uint32),
                ("observable_launches", ctypes.c_uint32)]


class sv_tune(ctypes.Structure):
    _fields_ = [("L", ctypes.c_uint8 * 41), ("k", ctypes.c_uint8 * 41)]


class sv_batch_info(ctypes.Structure):
    _fields_ = [("n_circuits", ctypes.c_uint32), ("n_programs", ctypes.c_uint32), ("n_resident", ctypes.c_uint32),
                ("total_params", ctypes.c_uint32), ("workspace_bytes", ctypes.c_uint64),
                ("smem_bytes", ctypes.c_uint32), ("grid", ctypes.c_uint32), ("graph", ctypes.c_uint32),
                ("pad", ctypes.c_uint32), ("last_ms", ctypes.c_double)]


assert ctypes.sizeof(sv_gate) == 40

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
lib = ctypes.CDLL(LIB_PATH)

_vp, _u32, _u64, _i32, _dp = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "sv_last_error": ([], ctypes.c_char_p),
    "sv_create": ([_u32, ctypes.c_int, _vp, _vp, ctypes.POINTER(_vp)], ctypes.c_int),
    "sv_destroy": ([_vp], ctypes.c_int),
    "sv_info": ([_vp, ctypes.POINTER(_u32), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_vp)], ctypes.c_int),
    "sv_reset_zero": ([_vp], ctypes.c_int),
    "sv_set_state": ([_vp, _vp], ctypes.c_int),
    "sv_get_state": ([_vp, _vp], ctypes.c_int),
    "sv_set_state_host": ([_vp, _vp], ctypes.c_int),
    "sv_get_state_host": ([_vp, _vp], ctypes.c_int),
    "sv_synchronize": ([_vp], ctypes.c_int),
    "sv_last_run_info": ([_vp, ctypes.POINTER(sv_run_info)], ctypes.c_int),
    "sv_partition": ([ctypes.POINTER(sv_circuit), _u32, ctypes.POINTER(_vp)], ctypes.c_int),
    "sv_partition_ex": ([ctypes.POINTER(sv_circuit), _u32, _u32, ctypes.POINTER(_vp)], ctypes.c_int),
    "sv_partition_gemm": ([ctypes.POINTER(sv_circuit), _u32, ctypes.POINTER(_vp)], ctypes.c_int),
    "sv_plan_stages": ([_vp, ctypes.POINTER(_u32), ctypes.POINTER(_u64), ctypes.POINTER(_u32)], ctypes.c_int),
    "sv_partition_hier": ([ctypes.POINTER(sv_circuit), _u32, ctypes.POINTER(_vp)], ctypes.c_int),
    "sv_hier_plan_info": ([_vp, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.POINTER(_u32), ctypes.POINTER(_u32)],
                          ctypes.c_int),
    "sv_gemm_plan_info": ([_vp, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.POINTER(_u32),
                           ctypes.POINTER(_u32), ctypes.POINTER(_u32), ctypes.POINTER(_u32),
                           ctypes.POINTER(ctypes.c_uint8)], ctypes.c_int),
    "sv_pauli_plan_info": ([_u32, ctypes.c_int, ctypes.POINTER(sv_observable), ctypes.POINTER(_u32),
                            ctypes.POINTER(_u64), ctypes.POINTER(_u64), ctypes.POINTER(_u32)], ctypes.c_int),
    "sv_plan_order": ([_vp, ctypes.POINTER(_u32), ctypes.POINTER(_u32)], ctypes.c_int),
    "sv_plan_centrality": ([_vp, ctypes.POINTER(_u32), ctypes.POINTER(_u64), ctypes.POINTER(_u32)], ctypes.c_int),
    "sv_plan_destroy": ([_vp], ctypes.c_int),
    "sv_plan_compile": ([_vp, _dp, _u32, ctypes.POINTER(_u32)], ctypes.c_int),
    "sv_permute_plan_info": ([_u32, ctypes.c_int, ctypes.POINTER(_u32), ctypes.POINTER(_u32), ctypes.POINTER(ctypes.c_uint64),
                              ctypes.POINTER(_u32), ctypes.POINTER(_u32)], ctypes.c_int),
    "sv_pauli_compile": ([_u32, ctypes.c_int, ctypes.POINTER(sv_observable), ctypes.POINTER(_u32)], ctypes.c_int),
    "sv_jit_stats": ([ctypes.POINTER(_u64), ctypes.POINTER(_u64), _dp], ctypes.c_int),
    "sv_qasm_parse": ([ctypes.c_char_p, ctypes.POINTER(sv_gate), _u32, ctypes.POINTER(_u32), ctypes.POINTER(_u32)],
                      ctypes.c_int),
    "sv_run": ([_vp, _vp, _dp, ctypes.c_int], ctypes.c_int),
    "sv_permute": ([_vp, ctypes.POINTER(_u32)], ctypes.c_int),
    "sv_expval": ([_vp, ctypes.POINTER(sv_observable), _dp], ctypes.c_int),
    "sv_norm": ([_vp, _dp], ctypes.c_int),
    "sv_norm_noalloc": ([_vp, _u32, ctypes.c_int, _vp, _vp], ctypes.c_int),
    "sv_grad": ([_vp, _vp, _dp, ctypes.POINTER(sv_observable), _dp, _dp], ctypes.c_int),
    "sv_timing_enable": ([_vp, ctypes.c_int], ctypes.c_int),
    "sv_timing_read": ([_vp, ctypes.POINTER(sv_timing), ctypes.c_int], ctypes.c_int),
    "sv_batch_create": ([ctypes.POINTER(sv_circuit), ctypes.POINTER(sv_observable), _u32, ctypes.POINTER(sv_tune), _vp,
                         ctypes.POINTER(_vp)], ctypes.c_int),
    "sv_run_batch": ([_vp, _dp, _dp, _dp], ctypes.c_int),
    "sv_autotune": ([_vp, _dp, ctypes.POINTER(sv_tune)], ctypes.c_int),
    "sv_batch_info_get": ([_vp, ctypes.POINTER(sv_batch_info)], ctypes.c_int),
    "sv_batch_destroy": ([_vp], ctypes.c_int),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def check(status):
    if status != SV_OK:
        raise SvError(status, lib.sv_last_error().decode())


def exported_symbols():
    return sorted(_SIGS)


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
_GATE_DTYPE = np.dtype([("kind", np.uint16), ("nq", np.uint8), ("q", np.uint8, 3), ("reserved", np.uint16),
                        ("param", np.int32), ("angle", np.float64, 3)], align=True)
assert _GATE_DTYPE.itemsize == ctypes.sizeof(sv_gate)


def gate_array(circuit):
    """sv_gate[] of a circuit (filled through one structured numpy array; the ctypes
    array shares its memory and keeps it alive)."""
    rows = []
    for g in circuit.gates:
        q = tuple(g.qubits) + (0,) * (3 - len(g.qubits))
        a = tuple(g.angles) + (0.0,) * (3 - len(g.angles))
        rows.append((GATE_CODES[g.kind], len(g.qubits), q, 0, g.param, a))
    buf = np.array(rows, dtype=_GATE_DTYPE) if rows else np.zeros(1, dtype=_GATE_DTYPE)
    arr = (sv_gate * len(buf)).from_buffer(buf)
    arr._keep = buf
    return arr


def circuit_struct(circuit):
    arr = gate_array(circuit)
    c = sv_circuit(circuit.n_qubits, len(circuit.gates), circuit.n_params,
                   ctypes.cast(arr, ctypes.POINTER(sv_gate)))
    return c, arr


def observable_struct(obs):
    n = obs.n_qubits
    codes = np.zeros((len(obs.terms), n), dtype=np.uint8)
    coeff = np.zeros(len(obs.terms), dtype=np.float64)
    for t, (c, s) in enumerate(obs.terms):
        coeff[t] = c
        for q, ch in enumerate(s):
            codes[t, q] = PAULI_CODES[ch]
    codes = np.ascontiguousarray(codes)
    o = sv_observable(len(obs.terms), n, codes.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                      coeff.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return o, (codes, coeff)


def as_double_ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
