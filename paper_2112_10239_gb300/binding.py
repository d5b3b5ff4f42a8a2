"""ctypes binding of ``libtlq.so`` (C-ABI in ``include/tlq.h``).

Argument marshalling only: every step of the computation runs in the CUDA library.
The module-level functions carry the C names (``tlq_init``, ``tlq_circuit_create``,
``tlq_expectation``, ...); ``Context`` / ``Circuit`` / ``Hamiltonian`` are thin owners
of the handles for Python callers. If the library is missing, importing this module
raises -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtlq.so")

TLQ_OK, TLQ_EINVAL, TLQ_ENOMEM, TLQ_EAGAIN, TLQ_ETIMEOUT, TLQ_ECUDA, TLQ_EKERNEL, TLQ_EUNSUPPORTED = range(8)
STATUS_NAMES = ["TLQ_OK", "TLQ_EINVAL", "TLQ_ENOMEM", "TLQ_EAGAIN", "TLQ_ETIMEOUT", "TLQ_ECUDA",
                "TLQ_EKERNEL", "TLQ_EUNSUPPORTED"]
TLQ_FP32, TLQ_MIXED_TC, TLQ_FP64_REF = 0, 1, 2
TLQ_PATH_CONE, TLQ_PATH_DENSE = 0, 1

# exported symbols declared in include/tlq.h
SYMBOLS = ["tlq_init", "tlq_destroy", "tlq_circuit_create", "tlq_circuit_destroy",
           "tlq_hamiltonian_create", "tlq_hamiltonian_destroy", "tlq_expectation",
           "tlq_expectation_grad", "tlq_expectation_grad_dev", "tlq_submit", "tlq_poll",
           "tlq_last_error", "tlq_plan_info", "tlq_plan_cone_stats", "tlq_profile_enable",
           "tlq_profile_last", "tlq_serving_stats", "tlq_version", "tlq_expectation_grad_static",
           "tlq_plan_dense_info", "tlq_plan_dense_bytes", "tlq_partial_trace_dev", "tlq_reduced_density",
           "tlq_mps_expectation_grad", "tlq_mps_expectation_grad_dev", "tlq_plan_mps_info"]


class tlq_gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("q0", ctypes.c_int32), ("q1", ctypes.c_int32),
                ("param", ctypes.c_int32), ("angle", ctypes.c_double)]


class tlq_term(ctypes.Structure):
    _fields_ = [("coeff", ctypes.c_double), ("nsites", ctypes.c_int32),
                ("sites", ctypes.POINTER(ctypes.c_int32)), ("paulis", ctypes.c_char_p)]


class tlq_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("mem_budget", ctypes.c_size_t), ("max_slots", ctypes.c_int),
                ("default_prec", ctypes.c_int), ("fuse_k", ctypes.c_int)]


class TLQError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load libtlq.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"{LIB_PATH} not built: run paper_2112_10239_gb300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)
        L.tlq_init.argtypes = [ctypes.POINTER(tlq_config), ctypes.POINTER(vp)]
        L.tlq_destroy.argtypes = [vp]
        L.tlq_circuit_create.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(tlq_gate), ctypes.c_int32,
                                         ctypes.c_int32, ctypes.POINTER(vp)]
        L.tlq_circuit_destroy.argtypes = [vp]
        L.tlq_hamiltonian_create.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(tlq_term), ctypes.c_int32,
                                             ctypes.POINTER(vp)]
        L.tlq_hamiltonian_destroy.argtypes = [vp]
        L.tlq_expectation.argtypes = [vp, vp, vp, dp, ctypes.c_int32, ctypes.c_int, dp]
        L.tlq_expectation_grad.argtypes = [vp, vp, vp, dp, ctypes.c_int32, ctypes.c_int, dp, dp]
        L.tlq_expectation_grad_dev.argtypes = [vp, vp, vp, vp, ctypes.c_int32, ctypes.c_int, vp, vp, vp]
        L.tlq_submit.argtypes = [vp, vp, vp, dp, ctypes.c_int32, ctypes.c_int, ctypes.c_int, dp, dp,
                                 ctypes.POINTER(ctypes.c_uint64)]
        L.tlq_poll.argtypes = [vp, ctypes.c_uint64, ctypes.c_int64]
        L.tlq_last_error.argtypes = [vp]
        L.tlq_last_error.restype = ctypes.c_char_p
        L.tlq_plan_info.argtypes = [vp, vp, vp, ip, ip, ip, ip]
        L.tlq_plan_cone_stats.argtypes = [vp, vp, vp, ip, ip, ip, ip, ip, ip, ip, ip]
        L.tlq_plan_dense_info.argtypes = [vp, vp, vp, ip, ip, ip, ip, ip, ip]
        L.tlq_plan_dense_bytes.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        L.tlq_partial_trace_dev.argtypes = [vp, vp, ctypes.c_int32, ip, ctypes.c_int32, vp, vp]
        L.tlq_reduced_density.argtypes = [vp, vp, dp, ip, ctypes.c_int32, dp]
        L.tlq_mps_expectation_grad.argtypes = [vp, vp, vp, dp, ctypes.c_int32, ctypes.c_int, dp, dp]
        L.tlq_mps_expectation_grad_dev.argtypes = [vp, vp, vp, vp, ctypes.c_int32, ctypes.c_int, vp, vp, vp]
        L.tlq_plan_mps_info.argtypes = [vp, vp, vp, ip, ctypes.POINTER(ctypes.c_int64), dp, dp]
        L.tlq_profile_enable.argtypes = [vp, ctypes.c_int]
        L.tlq_profile_last.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ip]
        L.tlq_expectation_grad_static.argtypes = [vp, vp, vp, vp, ctypes.c_int32, vp, vp, vp]
        L.tlq_serving_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), dp, dp, dp]
        L.tlq_version.argtypes = []
        L.tlq_version.restype = ctypes.c_int32
        for name in SYMBOLS:
            if name not in ("tlq_last_error", "tlq_version"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(status, ctx=None):
    if status != TLQ_OK:
        msg = lib().tlq_last_error(ctx)
        raise TLQError(status, msg.decode() if msg else "")
    return status


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---- C-named entry points -----------------------------------------------------------------

def tlq_init(device=0, mem_budget=0, max_slots=0, default_prec=TLQ_FP32):
    cfg = tlq_config(device, mem_budget, max_slots, default_prec, 0)
    h = ctypes.c_void_p()
    _check(lib().tlq_init(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def tlq_destroy(ctx):
    return _check(lib().tlq_destroy(ctx))


GATE_DTYPE = np.dtype([("kind", "<i4"), ("q0", "<i4"), ("q1", "<i4"), ("param", "<i4"), ("angle", "<f8")])


def gate_array(gates):
    """Gate tuples -> a contiguous array laid out as tlq_gate (kept alive by the caller)."""
    arr = np.array([tuple(g) for g in gates] if len(gates) else [(0, 0, -1, -1, 0.0)], dtype=GATE_DTYPE)
    assert arr.itemsize == ctypes.sizeof(tlq_gate)
    return arr


def tlq_circuit_create(ctx, n, gates, n_params):
    arr = gate_array(gates)
    h = ctypes.c_void_p()
    _check(lib().tlq_circuit_create(ctx, n, arr.ctypes.data_as(ctypes.POINTER(tlq_gate)), len(gates), n_params,
                                    ctypes.byref(h)), ctx)
    return h


def tlq_circuit_destroy(c):
    return _check(lib().tlq_circuit_destroy(c))


TERM_DTYPE = np.dtype([("coeff", "<f8"), ("nsites", "<i4"), ("pad", "<i4"), ("sites", "<u8"), ("paulis", "<u8")])


def term_array(terms):
    """Term tuples -> an array laid out as tlq_term plus the flat site/letter arrays its
    pointers refer to (the caller keeps all three alive for the call)."""
    T = max(1, len(terms))
    counts = np.array([len(s) for _, s, _ in terms] or [0], dtype=np.int64)
    flat_sites = np.array([x for _, s, _ in terms for x in s] or [0], dtype=np.int32)
    flat_letters = np.frombuffer(("".join(l for _, _, l in terms) or "Z").encode(), dtype=np.uint8).copy()
    off = np.zeros(T, dtype=np.int64)
    if len(terms) > 1:
        off[1:] = np.cumsum(counts)[:-1]
    arr = np.zeros(T, dtype=TERM_DTYPE)
    if len(terms):
        arr["coeff"] = [float(c) for c, _, _ in terms]
        arr["nsites"] = counts
        arr["sites"] = flat_sites.ctypes.data + 4 * off
        arr["paulis"] = flat_letters.ctypes.data + off
    assert arr.itemsize == ctypes.sizeof(tlq_term)
    return arr, (flat_sites, flat_letters)


def tlq_hamiltonian_create(ctx, n, terms):
    arr, keep = term_array(terms)
    h = ctypes.c_void_p()
    _check(lib().tlq_hamiltonian_create(ctx, n, arr.ctypes.data_as(ctypes.POINTER(tlq_term)), len(terms),
                                        ctypes.byref(h)), ctx)
    del keep
    return h


def tlq_hamiltonian_destroy(h):
    return _check(lib().tlq_hamiltonian_destroy(h))


def tlq_expectation(ctx, circ, ham, theta, prec=TLQ_FP32):
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    if theta.ndim == 1:
        theta = theta[None, :]
    B = theta.shape[0]
    E = np.zeros(B, dtype=np.float64)
    _check(lib().tlq_expectation(ctx, circ, ham, _dptr(theta), B, prec, _dptr(E)), ctx)
    return E


def tlq_expectation_grad(ctx, circ, ham, theta, prec=TLQ_FP32):
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    if theta.ndim == 1:
        theta = theta[None, :]
    B, P = theta.shape
    E = np.zeros(B, dtype=np.float64)
    G = np.zeros((B, P), dtype=np.float64)
    _check(lib().tlq_expectation_grad(ctx, circ, ham, _dptr(theta), B, prec, _dptr(E), _dptr(G)), ctx)
    return E, G


def tlq_expectation_grad_dev(ctx, circ, ham, theta_ptr, B, prec, energy_ptr, grad_ptr, stream_ptr):
    """Device-pointer call: every pointer is an int address on the context's device."""
    return _check(lib().tlq_expectation_grad_dev(ctx, circ, ham, ctypes.c_void_p(theta_ptr), B, prec,
                                                 ctypes.c_void_p(energy_ptr),
                                                 ctypes.c_void_p(grad_ptr) if grad_ptr else None,
                                                 ctypes.c_void_p(stream_ptr) if stream_ptr else None), ctx)


def tlq_mps_expectation(ctx, circ, ham, theta, prec=TLQ_FP32, grad=True):
    """Exact MPS route, host arrays: E [B] (and G [B, n_params] when grad) for theta [B, n_params]."""
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    if theta.ndim == 1:
        theta = theta[None, :]
    B, P = theta.shape
    E = np.zeros(B, dtype=np.float64)
    G = np.zeros((B, P), dtype=np.float64) if grad else None
    _check(lib().tlq_mps_expectation_grad(ctx, circ, ham, _dptr(theta), B, prec, _dptr(E),
                                          _dptr(G) if grad else None), ctx)
    return E, G


def tlq_mps_expectation_grad_dev(ctx, circ, ham, theta_ptr, B, prec, energy_ptr, grad_ptr, stream_ptr):
    """Exact MPS route, device pointers (int addresses); grad_ptr may be 0 for energies only."""
    return _check(lib().tlq_mps_expectation_grad_dev(ctx, circ, ham, ctypes.c_void_p(theta_ptr), B, prec,
                                                     ctypes.c_void_p(energy_ptr),
                                                     ctypes.c_void_p(grad_ptr) if grad_ptr else None,
                                                     ctypes.c_void_p(stream_ptr) if stream_ptr else None), ctx)


def tlq_plan_mps_info(ctx, circ, ham):
    """(max_bond_bits, complex entries per set, energy flops per set, energy+gradient flops per set)."""
    bits, el = ctypes.c_int32(), ctypes.c_int64()
    fe, fg = ctypes.c_double(), ctypes.c_double()
    _check(lib().tlq_plan_mps_info(ctx, circ, ham, ctypes.byref(bits), ctypes.byref(el), ctypes.byref(fe),
                                   ctypes.byref(fg)), ctx)
    return bits.value, el.value, fe.value, fg.value


def tlq_expectation_grad_static(ctx, circ, ham, theta_ptr, B, energy_ptr, grad_ptr, stream_ptr):
    """Allocation-free device-pointer call (scratch from the library's static array)."""
    return _check(lib().tlq_expectation_grad_static(ctx, circ, ham, ctypes.c_void_p(theta_ptr), B,
                                                    ctypes.c_void_p(energy_ptr),
                                                    ctypes.c_void_p(grad_ptr) if grad_ptr else None,
                                                    ctypes.c_void_p(stream_ptr) if stream_ptr else None), ctx)


def tlq_submit(ctx, circ, ham, theta, energy, grad, prec=TLQ_FP32):
    """Enqueue a request. ``theta``/``energy``/``grad`` are numpy arrays the caller keeps
    alive until tlq_poll returns TLQ_OK (grad may be None)."""
    B = theta.shape[0]
    t = ctypes.c_uint64()
    _check(lib().tlq_submit(ctx, circ, ham, _dptr(theta), B, 1 if grad is not None else 0, prec, _dptr(energy),
                            _dptr(grad) if grad is not None else None, ctypes.byref(t)), ctx)
    return t.value


def tlq_poll(ctx, ticket, timeout_us=0):
    """Returns the raw status (TLQ_OK, TLQ_EAGAIN, TLQ_ETIMEOUT) or raises on failure."""
    s = lib().tlq_poll(ctx, ticket, timeout_us)
    if s in (TLQ_OK, TLQ_EAGAIN, TLQ_ETIMEOUT):
        return s
    return _check(s, ctx)


def tlq_plan_info(ctx, circ, ham, n_terms):
    path = ctypes.c_int32()
    lo = np.zeros(n_terms, dtype=np.int32)
    w = np.zeros(n_terms, dtype=np.int32)
    ng = np.zeros(n_terms, dtype=np.int32)
    ip = ctypes.POINTER(ctypes.c_int32)
    _check(lib().tlq_plan_info(ctx, circ, ham, ctypes.byref(path), lo.ctypes.data_as(ip), w.ctypes.data_as(ip),
                               ng.ctypes.data_as(ip)), ctx)
    return path.value, lo, w, ng


def tlq_plan_cone_stats(ctx, circ, ham, n_terms):
    """Per work cone: (nrot, ndiag, npdiag, weff, wtrue, nterms, split), arrays of length ncones."""
    ip = ctypes.POINTER(ctypes.c_int32)
    nc = ctypes.c_int32()
    out = [np.zeros(max(1, n_terms), dtype=np.int32) for _ in range(7)]
    _check(lib().tlq_plan_cone_stats(ctx, circ, ham, ctypes.byref(nc), *[a.ctypes.data_as(ip) for a in out]), ctx)
    return tuple(a[:nc.value] for a in out)


def tlq_plan_dense_info(ctx, circ, ham):
    """(n_eff, n_passes, n_fwd_passes, n_rev_store, n_xterms, fused) of the dense plan."""
    v = [ctypes.c_int32() for _ in range(6)]
    _check(lib().tlq_plan_dense_info(ctx, circ, ham, *[ctypes.byref(x) for x in v]), ctx)
    return tuple(x.value for x in v)


def tlq_plan_dense_bytes(ctx, circ, ham, want_grad, prec=TLQ_FP32):
    """HBM bytes of one dense-path evaluation's pass schedule (see include/tlq.h)."""
    b = ctypes.c_double()
    _check(lib().tlq_plan_dense_bytes(ctx, circ, ham, 1 if want_grad else 0, prec, ctypes.byref(b)), ctx)
    return b.value


def tlq_partial_trace_dev(ctx, psi_ptr, n, keep, rho_ptr, stream_ptr=None):
    """Device-pointer partial trace: psi_ptr -> 2^n complex64, rho_ptr -> 2^m x 2^m complex64."""
    k = np.ascontiguousarray(keep, dtype=np.int32)
    _check(lib().tlq_partial_trace_dev(ctx, psi_ptr, n, k.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(k),
                                       rho_ptr, stream_ptr), ctx)


def tlq_reduced_density(ctx, circ, theta, keep):
    """rho_A (complex128 [2^m, 2^m]) of the circuit's output state for one parameter set."""
    k = np.ascontiguousarray(keep, dtype=np.int32)
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1)
    rho = np.zeros((1 << len(k), 1 << len(k)), dtype=np.complex128)
    _check(lib().tlq_reduced_density(ctx, circ, _dptr(th) if th.size else None,
                                     k.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(k),
                                     _dptr(rho.view(np.float64))), ctx)
    return rho


def tlq_profile_enable(ctx, on=True):
    return _check(lib().tlq_profile_enable(ctx, 1 if on else 0), ctx)


def tlq_profile_last(ctx):
    ms = ctypes.c_float()
    n = ctypes.c_int32()
    _check(lib().tlq_profile_last(ctx, ctypes.byref(ms), ctypes.byref(n)), ctx)
    return ms.value, n.value


def tlq_serving_stats(ctx):
    n = ctypes.c_int64()
    p50, p99, mb = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().tlq_serving_stats(ctx, ctypes.byref(n), ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(mb)), ctx)
    return n.value, p50.value, p99.value, mb.value


def tlq_version():
    return lib().tlq_version()


# ---- handle owners -------------------------------------------------------------------------

class Context:
    def __init__(self, device=0, mem_budget=0, max_slots=0, default_prec=TLQ_FP32):
        self.h = tlq_init(device, mem_budget, max_slots, default_prec)

    def close(self):
        if self.h:
            tlq_destroy(self.h)
            self.h = None

    def circuit(self, n, gates, n_params):
        return Circuit(self, n, gates, n_params)

    def hamiltonian(self, n, terms):
        return Hamiltonian(self, n, terms)

    def problem(self, prob):
        """(Circuit, Hamiltonian) for a workloads.Problem."""
        return self.circuit(prob.n, prob.gates, prob.n_params), self.hamiltonian(prob.n, prob.terms)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Circuit:
    def __init__(self, ctx, n, gates, n_params):
        self.ctx, self.n, self.n_params = ctx, n, n_params
        self.h = tlq_circuit_create(ctx.h, n, gates, n_params)

    def close(self):
        if self.h and self.ctx.h:
            tlq_circuit_destroy(self.h)
        self.h = None


class Hamiltonian:
    def __init__(self, ctx, n, terms):
        self.ctx, self.n, self.n_terms = ctx, n, len(terms)
        self.h = tlq_hamiltonian_create(ctx.h, n, terms)

    def close(self):
        if self.h and self.ctx.h:
            tlq_hamiltonian_destroy(self.h)
        self.h = None
