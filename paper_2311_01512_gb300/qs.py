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
QS_ARITH_FX = 2

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
    "qs_test_fail_allocations": (_I, [_I, _I]),
    "qs_test_set_error_word": (_I, [_P]),
    "qs_test_bounded_wait": (_I, [_P, ctypes.c_uint]),
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
    "qs_apply_pauli_channel": (_I, [_P, _I, _D, _D, _D]),
    "qs_apply_swap": (_I, [_P, _I, _I]),
    "qs_partial_trace": (_I, [_P, _IP, _I, _P, ctypes.POINTER(_P)]),
    "qs_expec_pauli_sum": (_I, [_P, _IP, _DP, _I, _DP]),
    "qs_calc_norm_or_trace": (_I, [_P, _DP]),
    "qs_synchronize": (_I, [_P]),
    "qs_record_begin": (_I, [_P]),
    "qs_record_end": (_I, [_P, ctypes.POINTER(_P)]),
    "qs_program_run": (_I, [_P]),
    "qs_program_destroy": (_I, [_P]),
    "qs_expec_pauli_sum_noalloc": (_I, [_P, _I, _I, _I, _IP, _DP, _I, _P, _DP]),
    "qs_circuit_create": (_I, [_I, ctypes.POINTER(_P)]),
    "qs_circuit_destroy": (_I, [_P]),
    "qs_circuit_add_unitary": (_I, [_P, _IP, _I, _IP, _I, _DP]),
    "qs_circuit_add_diagonal": (_I, [_P, _IP, _I, _DP]),
    "qs_circuit_add_pauli_gadget": (_I, [_P, _IP, _IP, _I, _D]),
    "qs_circuit_plan": (_I, [_P, _I, _I]),
    "qs_circuit_get_plan": (_I, [_P, _IP, _IP, _IP]),
    "qs_circuit_apply": (_I, [_P, _P]),
    "qs_apply_dense_block": (_I, [_P, _IP, _I, _DP]),
    "qs_costmodel_create": (_I, [ctypes.c_ulonglong, ctypes.POINTER(_P)]),
    "qs_costmodel_destroy": (_I, [_P]),
    "qs_costmodel_get_params": (_I, [_P, ctypes.POINTER(ctypes.c_float), _I]),
    "qs_costmodel_set_params": (_I, [_P, ctypes.POINTER(ctypes.c_float), _I]),
    "qs_costmodel_encode": (_I, [_I, _I, ctypes.c_ulonglong, _I, _I, _P, ctypes.POINTER(ctypes.c_float)]),
    "qs_costmodel_predict": (_I, [_P, ctypes.POINTER(ctypes.c_float), _I, ctypes.POINTER(ctypes.c_float)]),
    "qs_costmodel_gradient": (_I, [_P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), _I,
                                   ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
    "qs_costmodel_train": (_I, [_P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), _I, _I, _I,
                                ctypes.c_float, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_float)]),
    "qs_circuit_plan_cost": (_I, [_P, _P, _P, _I, _I]),
    "qs_circuit_plan_relabel": (_I, [_P, _P, _P, _I, ctypes.c_double]),
    "qs_circuit_get_relabel": (_I, [_P, _IP]),
    "qs_batch_create": (_I, [_I, _IP, _I, _P, ctypes.POINTER(_P)]),
    "qs_batch_create_mixed": (_I, [_I, _IP, _IP, _I, _P, ctypes.POINTER(_P)]),
    "qs_batch_add_kraus": (_I, [_P, _I, _IP, _I, _DP, _I]),
    "qs_batch_add_dephasing": (_I, [_P, _I, _I, _D]),
    "qs_batch_add_two_qubit_dephasing": (_I, [_P, _I, _I, _I, _D]),
    "qs_batch_add_depolarising": (_I, [_P, _I, _I, _D]),
    "qs_batch_add_two_qubit_depolarising": (_I, [_P, _I, _I, _I, _D]),
    "qs_batch_add_damping": (_I, [_P, _I, _I, _D]),
    "qs_batch_add_pauli_channel": (_I, [_P, _I, _I, _D, _D, _D]),
    "qs_batch_destroy": (_I, [_P]),
    "qs_batch_pool_amps": (_I, [_P, ctypes.POINTER(_S)]),
    "qs_batch_state_offset": (_I, [_P, _I, ctypes.POINTER(_S)]),
    "qs_batch_bind_pool": (_I, [_P, _P]),
    "qs_batch_add_unitary": (_I, [_P, _I, _IP, _I, _IP, _I, _DP]),
    "qs_batch_add_diagonal": (_I, [_P, _I, _IP, _I, _DP]),
    "qs_batch_add_pauli_gadget": (_I, [_P, _I, _IP, _IP, _I, _D]),
    "qs_batch_compile": (_I, [_P, _I]),
    "qs_batch_run": (_I, [_P]),
    "qs_batch_info": (_I, [_P, _IP, _IP, _IP, ctypes.POINTER(ctypes.c_long)]),
}

QS_COST_FEATURES = 64
QS_COST_PARAMS = 8385
QS_COST_FUSED_DENSE, QS_COST_GATE1, QS_COST_DENSE, QS_COST_DIAGONAL, QS_COST_GADGET, QS_COST_PHASE = range(6)

QS_PLAN_NONE = 0
QS_PLAN_GREEDY = 1
QS_PLAN_COST = 2

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


def qs_apply_swap(h, t1, t2):
    _check(_lib.qs_apply_swap(h, int(t1), int(t2)), "qs_apply_swap")


def qs_apply_pauli_channel(h, t, px, py, pz):
    _check(_lib.qs_apply_pauli_channel(h, int(t), float(px), float(py), float(pz)), "qs_apply_pauli_channel")


def qs_partial_trace(h, targs, d_out):
    t, nt = _ints(targs)
    out = _P()
    _check(_lib.qs_partial_trace(h, t, nt, _P(d_out), ctypes.byref(out)), "qs_partial_trace")
    return out


def _check_paulis(p, c, num_qubits, name):
    """The C side reads paulis[n * num_qubits + q]: the array must be T x N."""
    if c.ndim != 1 or p.shape != (c.shape[0], num_qubits):
        raise ValueError("%s: paulis must have shape (len(coeffs), num_qubits) = (%d, %d), got %s"
                         % (name, c.shape[0] if c.ndim == 1 else -1, num_qubits, p.shape))


def qs_expec_pauli_sum(h, paulis, coeffs):
    p = np.ascontiguousarray(np.asarray(paulis, dtype=np.int32))
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    nq = ctypes.c_int()
    _check(_lib.qs_get_info(h, ctypes.byref(nq), None, None, None), "qs_get_info")
    _check_paulis(p, c, nq.value, "qs_expec_pauli_sum")
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
    _check_paulis(p, c, num_qubits, "qs_expec_pauli_sum_noalloc")
    out = (ctypes.c_double * 2)()
    _check(_lib.qs_expec_pauli_sum_noalloc(_P(d_amps), num_qubits, 1 if is_density else 0, prec,
                                           p.ctypes.data_as(_IP), c.ctypes.data_as(_DP), c.shape[0],
                                           _P(stream), out), "qs_expec_pauli_sum_noalloc")
    return complex(out[0], out[1])


def qs_test_fail_allocations(skip, count):
    """Test hook: the next `skip` library allocations succeed, the `count`
    after them fail on the host (see include/qs.h)."""
    _check(_lib.qs_test_fail_allocations(int(skip), int(count)), "qs_test_fail_allocations")


def qs_test_set_error_word(h):
    """Test hook: set the handle's device error word (the next
    qs_synchronize reports QS_ERR_TIMEOUT once)."""
    _check(_lib.qs_test_set_error_word(h), "qs_test_set_error_word")


def qs_test_bounded_wait(h, polls):
    """Test hook: a device wait that nothing ends runs out after `polls`
    polls and sets the handle's error word (see include/qs.h)."""
    _check(_lib.qs_test_bounded_wait(h, int(polls)), "qs_test_bounded_wait")


def qs_calc_norm_or_trace(h):
    out = (ctypes.c_double * 2)()
    _check(_lib.qs_calc_norm_or_trace(h, out), "qs_calc_norm_or_trace")
    return complex(out[0], out[1])


def qs_synchronize(h):
    _check(_lib.qs_synchronize(h), "qs_synchronize")


def qs_record_begin(h):
    _check(_lib.qs_record_begin(h), "qs_record_begin")


def qs_record_end(h):
    p = _P()
    _check(_lib.qs_record_end(h, ctypes.byref(p)), "qs_record_end")
    return p


def qs_program_run(p):
    _check(_lib.qs_program_run(p), "qs_program_run")


def qs_program_destroy(p):
    _check(_lib.qs_program_destroy(p), "qs_program_destroy")


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


class Circuit:
    """A recorded circuit (qs_circuit_*): unitary operation records from
    workloads.py, planned into fused blocks inside the library."""

    def __init__(self, num_qubits, ops=()):
        self.handle = _P()
        _check(_lib.qs_circuit_create(num_qubits, ctypes.byref(self.handle)), "qs_circuit_create")
        for op in ops:
            self.add(op)

    def add(self, op):
        kind = op["op"]
        if kind == "unitary":
            c, nc = _ints(op["ctrls"])
            t, nt = _ints(op["targs"])
            keep, mp = _doubles(op["mat"])
            _check(_lib.qs_circuit_add_unitary(self.handle, c, nc, t, nt, mp), "qs_circuit_add_unitary")
        elif kind == "diagonal":
            t, nt = _ints(op["targs"])
            keep, dp = _doubles(np.asarray(op["diag"], dtype=np.complex128))
            _check(_lib.qs_circuit_add_diagonal(self.handle, t, nt, dp), "qs_circuit_add_diagonal")
        elif kind == "gadget":
            t, nt = _ints(op["targs"])
            p, _ = _ints(op["paulis"])
            _check(_lib.qs_circuit_add_pauli_gadget(self.handle, t, p, nt, float(op["theta"])),
                   "qs_circuit_add_pauli_gadget")
        else:
            raise ValueError("circuits record unitary operations only, not " + kind)

    def plan(self, kind=QS_PLAN_GREEDY, max_block_qubits=5):
        _check(_lib.qs_circuit_plan(self.handle, int(kind), int(max_block_qubits)), "qs_circuit_plan")
        return self.stats()

    def stats(self):
        g, b, f = _I(), _I(), _I()
        _check(_lib.qs_circuit_get_plan(self.handle, ctypes.byref(g), ctypes.byref(b), ctypes.byref(f)),
               "qs_circuit_get_plan")
        return {"gates": g.value, "blocks": b.value, "fused": f.value}

    def plan_cost(self, model, state_handle, max_block_qubits=5, window=24):
        _check(_lib.qs_circuit_plan_cost(self.handle, model.handle, state_handle, int(max_block_qubits), int(window)),
               "qs_circuit_plan_cost")
        return self.stats()

    def plan_relabel(self, model, state_handle, low_qubits=5, swap_passes=1.2):
        """Lazy qubit relabelling of the current plan (see include/qs.h);
        returns the number of SWAP passes it adds."""
        _check(_lib.qs_circuit_plan_relabel(self.handle, model.handle, state_handle, int(low_qubits),
                                            float(swap_passes)), "qs_circuit_plan_relabel")
        n = _I()
        _check(_lib.qs_circuit_get_relabel(self.handle, ctypes.byref(n)), "qs_circuit_get_relabel")
        return n.value

    def apply(self, state_handle):
        _check(_lib.qs_circuit_apply(self.handle, state_handle), "qs_circuit_apply")

    def close(self):
        if getattr(self, "handle", None):
            _check(_lib.qs_circuit_destroy(self.handle), "qs_circuit_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """qs_batch_*: many statevectors (or density matrices, density[s] true,
    held as Choi vectors) with their own circuits in one persistent launch.
    The amplitude pool is a torch tensor owned by this object."""

    def __init__(self, num_qubits, prec=QS_C64, stream=None, device="cuda", density=None):
        import torch
        self.num_qubits = [int(q) for q in num_qubits]
        self.density = [bool(d) for d in density] if density is not None else [False] * len(self.num_qubits)
        self.storage_qubits = [2 * q if d else q for q, d in zip(self.num_qubits, self.density)]
        self.prec = prec
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        q, nq = _ints(self.num_qubits)
        dens, _ = _ints([1 if d else 0 for d in self.density])
        self.handle = _P()
        _check(_lib.qs_batch_create_mixed(nq, q, dens, prec, _P(self.stream.cuda_stream), ctypes.byref(self.handle)),
               "qs_batch_create_mixed")
        n = _S()
        _check(_lib.qs_batch_pool_amps(self.handle, ctypes.byref(n)), "qs_batch_pool_amps")
        dtype = torch.complex128 if prec == QS_C128 else torch.complex64
        self.pool = torch.zeros(n.value, dtype=dtype, device=device)
        _check(_lib.qs_batch_bind_pool(self.handle, _P(self.pool.data_ptr())), "qs_batch_bind_pool")
        self.offsets = []
        for s in range(len(self.num_qubits)):
            off = _S()
            _check(_lib.qs_batch_state_offset(self.handle, s, ctypes.byref(off)), "qs_batch_state_offset")
            self.offsets.append(off.value)

    def view(self, s):
        return self.pool[self.offsets[s]:self.offsets[s] + (1 << self.storage_qubits[s])]

    def add(self, s, op):
        kind = op["op"]
        if kind == "unitary":
            c, nc = _ints(op["ctrls"])
            t, nt = _ints(op["targs"])
            keep, mp = _doubles(op["mat"])
            _check(_lib.qs_batch_add_unitary(self.handle, s, c, nc, t, nt, mp), "qs_batch_add_unitary")
        elif kind == "diagonal":
            t, nt = _ints(op["targs"])
            keep, dp = _doubles(np.asarray(op["diag"], dtype=np.complex128))
            _check(_lib.qs_batch_add_diagonal(self.handle, s, t, nt, dp), "qs_batch_add_diagonal")
        elif kind == "gadget":
            t, nt = _ints(op["targs"])
            p, _ = _ints(op["paulis"])
            _check(_lib.qs_batch_add_pauli_gadget(self.handle, s, t, p, nt, float(op["theta"])),
                   "qs_batch_add_pauli_gadget")
        elif kind == "kraus":
            t, nt = _ints(op["targs"])
            k = np.ascontiguousarray(np.asarray(op["kraus"], dtype=np.complex128))
            keep, kp = _doubles(k)
            _check(_lib.qs_batch_add_kraus(self.handle, s, t, nt, kp, k.shape[0]), "qs_batch_add_kraus")
        elif kind in ("dephasing", "depolarising", "damping"):
            fn = getattr(_lib, "qs_batch_add_" + kind)
            _check(fn(self.handle, s, int(op["targs"][0]), float(op["p"])), "qs_batch_add_" + kind)
        elif kind in ("dephasing2", "depolarising2"):
            fn = getattr(_lib, "qs_batch_add_two_qubit_" + kind[:-1])
            _check(fn(self.handle, s, int(op["targs"][0]), int(op["targs"][1]), float(op["p"])),
                   "qs_batch_add_two_qubit_" + kind[:-1])
        elif kind == "pauli_channel":
            px, py, pz = (float(x) for x in op["probs"])
            _check(_lib.qs_batch_add_pauli_channel(self.handle, s, int(op["targs"][0]), px, py, pz),
                   "qs_batch_add_pauli_channel")
        else:
            raise ValueError("operation kind %r is not supported in batches" % kind)

    def compile(self, autotune=True):
        _check(_lib.qs_batch_compile(self.handle, 1 if autotune else 0), "qs_batch_compile")

    def run(self):
        _check(_lib.qs_batch_run(self.handle), "qs_batch_run")

    def info(self):
        a, b, c, d = _I(), _I(), _I(), ctypes.c_long()
        _check(_lib.qs_batch_info(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)),
               "qs_batch_info")
        return {"threads": a.value, "ctas": b.value, "smem_qubits": c.value, "total_ops": d.value}

    def close(self):
        if getattr(self, "handle", None):
            _check(_lib.qs_batch_destroy(self.handle), "qs_batch_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qs_apply_dense_block(h, targs, mat):
    t, nt = _ints(targs)
    keep, mp = _doubles(mat)
    _check(_lib.qs_apply_dense_block(h, t, nt, mp), "qs_apply_dense_block")


_FP = ctypes.POINTER(ctypes.c_float)


def _f32(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    return a, a.ctypes.data_as(_FP)


class CostModel:
    """Handle of the library's cost-model network (qs_costmodel_*)."""

    def __init__(self, seed=2311015120):
        self.handle = _P()
        _check(_lib.qs_costmodel_create(ctypes.c_ulonglong(seed), ctypes.byref(self.handle)), "qs_costmodel_create")

    def get_params(self):
        out = np.empty(QS_COST_PARAMS, dtype=np.float32)
        _check(_lib.qs_costmodel_get_params(self.handle, out.ctypes.data_as(_FP), QS_COST_PARAMS),
               "qs_costmodel_get_params")
        return out

    def set_params(self, params):
        keep, pp = _f32(params)
        _check(_lib.qs_costmodel_set_params(self.handle, pp, keep.size), "qs_costmodel_set_params")

    def predict(self, X):
        keep, xp = _f32(X)
        out = np.empty(keep.shape[0], dtype=np.float32)
        _check(_lib.qs_costmodel_predict(self.handle, xp, keep.shape[0], out.ctypes.data_as(_FP)),
               "qs_costmodel_predict")
        return out

    def gradient(self, X, t):
        kx, xp = _f32(X)
        kt, tp = _f32(t)
        g = np.empty(QS_COST_PARAMS, dtype=np.float32)
        loss = ctypes.c_float()
        _check(_lib.qs_costmodel_gradient(self.handle, xp, tp, kx.shape[0], g.ctypes.data_as(_FP), ctypes.byref(loss)),
               "qs_costmodel_gradient")
        return g, loss.value

    def train(self, X, t, epochs=200, batch=512, lr=1e-3, seed=7):
        kx, xp = _f32(X)
        kt, tp = _f32(t)
        loss = ctypes.c_float()
        _check(_lib.qs_costmodel_train(self.handle, xp, tp, kx.shape[0], int(epochs), int(batch), ctypes.c_float(lr),
                                       ctypes.c_ulonglong(seed), ctypes.byref(loss)), "qs_costmodel_train")
        return loss.value

    def close(self):
        if getattr(self, "handle", None):
            _check(_lib.qs_costmodel_destroy(self.handle), "qs_costmodel_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qs_costmodel_encode(kind, width, qmask, nctrl, weight, state_handle):
    out = np.empty(QS_COST_FEATURES, dtype=np.float32)
    _check(_lib.qs_costmodel_encode(int(kind), int(width), ctypes.c_ulonglong(int(qmask)), int(nctrl), int(weight),
                                    state_handle, out.ctypes.data_as(_FP)), "qs_costmodel_encode")
    return out


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
    elif kind == "pauli_channel":
        qs_apply_pauli_channel(h, op["targs"][0], *op["probs"])
    elif kind == "swap":
        qs_apply_swap(h, op["targs"][0], op["targs"][1])
    else:
        raise ValueError("unknown op " + kind)
