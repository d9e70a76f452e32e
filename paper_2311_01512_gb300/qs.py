"""Thin ctypes binding of the C ABI in include/qs.h.

Functions keep the C names and only marshal arguments: Python lists and numpy
arrays become C arrays, torch CUDA tensors provide device memory and streams.
Every operation runs in the CUDA library; there is no fallback.  Importing this
module raises if libqsim.so has not been built.
"""

import ctypes
import os

import numpy as np

from .build import LIB_PATH

if not os.path.exists(LIB_PATH):
    raise ImportError("libqsim.so is not built (%s); run __graft_entry__.build() on a machine with nvcc" % LIB_PATH)

_lib = ctypes.CDLL(LIB_PATH)

QS_C64 = 0
QS_C128 = 1
QS_ARITH_DF = 0
QS_ARITH_F64 = 1

STATUS = {
    0: "QS_OK", 1: "QS_ERR_ARG", 2: "QS_ERR_QUBIT_RANGE", 3: "QS_ERR_DUP_QUBIT",
    4: "QS_ERR_TARGET_IS_CTRL", 5: "QS_ERR_TOO_MANY_TARGETS", 6: "QS_ERR_NOT_DENSMATR",
    7: "QS_ERR_OOM", 8: "QS_ERR_CUDA", 9: "QS_ERR_TIMEOUT", 10: "QS_ERR_ALIGN",
}

# Every symbol declared in include/qs.h, with its ctypes signature.
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_S = ctypes.c_size_t
_IP = ctypes.POINTER(ctypes.c_int)
_DP = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "qs_status_str": (ctypes.c_char_p, [_I]),
    "qs_create_statevector": (_I, [_I, _I, _P, _P, ctypes.POINTER(_P)]),
    "qs_create_densmatr": (_I, [_I, _I, _P, _P, ctypes.POINTER(_P)]),
    "qs_destroy": (_I, [_P]),
    "qs_get_info": (_I, [_P, _IP, _IP, _IP, _IP]),
    "qs_device_ptr": (_I, [_P, ctypes.POINTER(_P)]),
    "qs_set_arithmetic": (_I, [_P, _I, _I]),
    "qs_set_tensor_cores": (_I, [_P, _I]),
    "qs_set_amps": (_I, [_P, _P, _S, _S]),
    "qs_get_amps": (_I, [_P, _P, _S, _S]),
    "qs_init_zero": (_I, [_P]),
    "qs_init_pure_densmatr": (_I, [_P, _P, _D, _I]),
    "qs_apply_ctrl_multi_target": (_I, [_P, _IP, _I, _IP, _I, _DP]),
    "qs_apply_diagonal": (_I, [_P, _IP, _I, _DP]),
    "qs_apply_pauli_gadget": (_I, [_P, _IP, _IP, _I, _D]),
    "qs_apply_kraus": (_I, [_P, _IP, _I, _DP, _I]),
    "qs_apply_dephasing": (_I, [_P, _I, _D]),
    "qs_apply_two_qubit_dephasing": (_I, [_P, _I, _I, _D]),
    "qs_apply_depolarising": (_I, [_P, _I, _D]),
    "qs_apply_two_qubit_depolarising": (_I, [_P, _I, _I, _D]),
    "qs_apply_damping": (_I, [_P, _I, _D]),
    "qs_partial_trace": (_I, [_P, _IP, _I, _P, ctypes.POINTER(_P)]),
    "qs_expec_pauli_sum": (_I, [_P, _IP, _DP, _I, _DP]),
    "qs_calc_norm_or_trace": (_I, [_P, _DP]),
    "qs_synchronize": (_I, [_P]),
    "qs_expec_pauli_sum_noalloc": (_I, [_P, _I, _I, _I, _IP, _DP, _I, _P, _DP]),
}

NOALLOC_MAX_TERMS = 256
for _name, (_res, _args) in SIGNATURES.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


class QSError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.qs_status_str(status).decode()
        super().__init__("%s: %s (%s)" % (where, STATUS.get(status, status), msg))


def _check(status, where):
    if status != 0:
        raise QSError(status, where)


def _ints(xs):
    xs = [int(x) for x in xs]
    return (ctypes.c_int * max(1, len(xs)))(*xs), len(xs)


def _doubles(arr):
    """complex or real array -> contiguous float64 buffer (kept alive by the caller)."""
    a = np.asarray(arr)
    if np.iscomplexobj(a):
        a = np.ascontiguousarray(a, dtype=np.complex128).view(np.float64)
    else:
        a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_DP)


def lib_path():
    return LIB_PATH


# --------------------------------------------------------------------------
# Raw C-ABI calls (same names as include/qs.h)
# --------------------------------------------------------------------------

def qs_create_statevector(num_qubits, prec, d_amps, stream):
    h = _P()
    _check(_lib.qs_create_statevector(num_qubits, prec, _P(d_amps), _P(stream), ctypes.byref(h)),
           "qs_create_statevector")
    return h


def qs_create_densmatr(num_qubits, prec, d_amps, stream):
    h = _P()
    _check(_lib.qs_create_densmatr(num_qubits, prec, _P(d_amps), _P(stream), ctypes.byref(h)),
           "qs_create_densmatr")
    return h


def qs_destroy(h):
    _check(_lib.qs_destroy(h), "qs_destroy")


def qs_set_amps(h, host_array, first=0):
    a = np.ascontiguousarray(host_array)
    _check(_lib.qs_set_amps(h, a.ctypes.data, first, a.shape[0]), "qs_set_amps")
    return a


def qs_set_amps_ptr(h, host_ptr, first, count):
    _check(_lib.qs_set_amps(h, _P(host_ptr), first, count), "qs_set_amps")


def qs_get_amps(h, out_array, first=0):
    _check(_lib.qs_get_amps(h, out_array.ctypes.data, first, out_array.shape[0]), "qs_get_amps")
    return out_array


def qs_set_arithmetic(h, arith, f64_share_16ths=0):
    _check(_lib.qs_set_arithmetic(h, int(arith), int(f64_share_16ths)), "qs_set_arithmetic")


def qs_set_tensor_cores(h, enable):
    _check(_lib.qs_set_tensor_cores(h, 1 if enable else 0), "qs_set_tensor_cores")


def qs_init_zero(h):
    _check(_lib.qs_init_zero(h), "qs_init_zero")


def qs_init_pure_densmatr(rho, psi, weight=1.0, accumulate=False):
    _check(_lib.qs_init_pure_densmatr(rho, psi, float(weight), 1 if accumulate else 0), "qs_init_pure_densmatr")


def qs_apply_ctrl_multi_target(h, ctrls, targs, mat):
    c, nc = _ints(ctrls)
    t, nt = _ints(targs)
    keep, mp = _doubles(mat)
    _check(_lib.qs_apply_ctrl_multi_target(h, c, nc, t, nt, mp), "qs_apply_ctrl_multi_target")


def qs_apply_diagonal(h, targs, diag):
    t, nt = _ints(targs)
    keep, dp = _doubles(np.asarray(diag, dtype=np.complex128))
    _check(_lib.qs_apply_diagonal(h, t, nt, dp), "qs_apply_diagonal")


def qs_apply_pauli_gadget(h, targs, paulis, theta):
    t, nt = _ints(targs)
    p, npl = _ints(paulis)
    if npl != nt:
        raise ValueError("targs and paulis differ in length")
    _check(_lib.qs_apply_pauli_gadget(h, t, p, nt, float(theta)), "qs_apply_pauli_gadget")


def qs_apply_kraus(h, targs, kraus):
    t, nt = _ints(targs)
    ks = np.ascontiguousarray(np.stack([np.asarray(k, dtype=np.complex128) for k in kraus]))
    keep, kp = _doubles(ks)
    _check(_lib.qs_apply_kraus(h, t, nt, kp, len(kraus)), "qs_apply_kraus")


def qs_apply_dephasing(h, t, p):
    _check(_lib.qs_apply_dephasing(h, int(t), float(p)), "qs_apply_dephasing")


def qs_apply_two_qubit_dephasing(h, t1, t2, p):
    _check(_lib.qs_apply_two_qubit_dephasing(h, int(t1), int(t2), float(p)), "qs_apply_two_qubit_dephasing")


def qs_apply_depolarising(h, t, p):
    _check(_lib.qs_apply_depolarising(h, int(t), float(p)), "qs_apply_depolarising")


def qs_apply_two_qubit_depolarising(h, t1, t2, p):
    _check(_lib.qs_apply_two_qubit_depolarising(h, int(t1), int(t2), float(p)), "qs_apply_two_qubit_depolarising")


def qs_apply_damping(h, t, p):
    _check(_lib.qs_apply_damping(h, int(t), float(p)), "qs_apply_damping")


def qs_partial_trace(h, targs, d_out):
    t, nt = _ints(targs)
    out = _P()
    _check(_lib.qs_partial_trace(h, t, nt, _P(d_out), ctypes.byref(out)), "qs_partial_trace")
    return out


def qs_expec_pauli_sum(h, paulis, coeffs):
    p = np.ascontiguousarray(np.asarray(paulis, dtype=np.int32))
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    out = (ctypes.c_double * 2)()
    _check(_lib.qs_expec_pauli_sum(h, p.ctypes.data_as(_IP), c.ctypes.data_as(_DP), c.shape[0], out),
           "qs_expec_pauli_sum")
    return complex(out[0], out[1])


def qs_expec_pauli_sum_noalloc(d_amps, num_qubits, is_density, prec, paulis, coeffs, stream):
    """Expectation value from a raw device pointer, with no allocation inside
    the library (see include/qs.h).  For callers that cannot allocate GPU
    memory; at most NOALLOC_MAX_TERMS terms."""
    p = np.ascontiguousarray(np.asarray(paulis, dtype=np.int32))
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    if c.shape[0] > NOALLOC_MAX_TERMS:
        raise ValueError("qs_expec_pauli_sum_noalloc takes at most %d terms, got %d" % (NOALLOC_MAX_TERMS, c.shape[0]))
    out = (ctypes.c_double * 2)()
    _check(_lib.qs_expec_pauli_sum_noalloc(_P(d_amps), num_qubits, 1 if is_density else 0, prec,
                                           p.ctypes.data_as(_IP), c.ctypes.data_as(_DP), c.shape[0],
                                           _P(stream), out), "qs_expec_pauli_sum_noalloc")
    return complex(out[0], out[1])


def qs_calc_norm_or_trace(h):
    out = (ctypes.c_double * 2)()
    _check(_lib.qs_calc_norm_or_trace(h, out), "qs_calc_norm_or_trace")
    return complex(out[0], out[1])


def qs_synchronize(h):
    _check(_lib.qs_synchronize(h), "qs_synchronize")


def qs_get_info(h):
    a, b, c, d = _I(), _I(), _I(), _I()
    _check(_lib.qs_get_info(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)), "qs_get_info")
    return a.value, b.value, c.value, d.value


# --------------------------------------------------------------------------
# torch-backed state objects: torch allocates device memory, the library
# computes.  The tensor is kept alive by the object.
# --------------------------------------------------------------------------

class State:
    """A statevector or density matrix (Choi vector) in a torch CUDA tensor."""

    def __init__(self, num_qubits, density=False, prec=QS_C128, stream=None, device="cuda", storage=None):
        import torch
        self.num_qubits = num_qubits
        self.density = density
        self.prec = prec
        self.storage_qubits = 2 * num_qubits if density else num_qubits
        dtype = torch.complex128 if prec == QS_C128 else torch.complex64
        if storage is None:
            storage = torch.empty(1 << self.storage_qubits, dtype=dtype, device=device)
        self.tensor = storage
        if stream is None:
            stream = torch.cuda.current_stream(self.tensor.device)
        self.stream = stream
        create = qs_create_densmatr if density else qs_create_statevector
        self.handle = create(num_qubits, prec, self.tensor.data_ptr(), stream.cuda_stream)

    @classmethod
    def wrap(cls, handle, tensor, num_qubits, density, prec, stream):
        obj = cls.__new__(cls)
        obj.num_qubits, obj.density, obj.prec = num_qubits, density, prec
        obj.storage_qubits = 2 * num_qubits if density else num_qubits
        obj.tensor, obj.stream, obj.handle = tensor, stream, handle
        return obj

    def close(self):
        if getattr(self, "handle", None):
            qs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def np_dtype(self):
        return np.complex128 if self.prec == QS_C128 else np.complex64

    def set_amps(self, host):
        return qs_set_amps(self.handle, np.asarray(host, dtype=self.np_dtype))

    def get_amps(self):
        out = np.empty(1 << self.storage_qubits, dtype=self.np_dtype)
        return qs_get_amps(self.handle, out)

    def partial_trace(self, targs):
        import torch
        m = self.num_qubits - len(targs)
        t = torch.empty(1 << (2 * m), dtype=self.tensor.dtype, device=self.tensor.device)
        h = qs_partial_trace(self.handle, targs, t.data_ptr())
        return State.wrap(h, t, m, True, self.prec, self.stream)


def apply_op(h, op):
    """Apply one operation record (see workloads.py) through the C ABI."""
    kind = op["op"]
    if kind == "unitary":
        qs_apply_ctrl_multi_target(h, op["ctrls"], op["targs"], op["mat"])
    elif kind == "diagonal":
        qs_apply_diagonal(h, op["targs"], op["diag"])
    elif kind == "gadget":
        qs_apply_pauli_gadget(h, op["targs"], op["paulis"], op["theta"])
    elif kind == "kraus":
        qs_apply_kraus(h, op["targs"], op["kraus"])
    elif kind == "dephasing":
        qs_apply_dephasing(h, op["targs"][0], op["p"])
    elif kind == "dephasing2":
        qs_apply_two_qubit_dephasing(h, op["targs"][0], op["targs"][1], op["p"])
    elif kind == "depolarising":
        qs_apply_depolarising(h, op["targs"][0], op["p"])
    elif kind == "depolarising2":
        qs_apply_two_qubit_depolarising(h, op["targs"][0], op["targs"][1], op["p"])
    elif kind == "damping":
        qs_apply_damping(h, op["targs"][0], op["p"])
    else:
        raise ValueError("unknown op " + kind)
