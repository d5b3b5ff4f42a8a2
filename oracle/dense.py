"""ctypes binding of the C oracle plus gradient routes built on the plain energy.

Test infrastructure only (see the package docstring).

Routes to the gradient (TensorLy-Quantum Sec. 3, the full gradient of <H>):
  * ``grad_adjoint``     -- the C oracle's own adjoint sweep;
  * ``grad_param_shift`` -- [E(theta_p + pi/2) - E(theta_p - pi/2)] / 2, exact when the
                            parameter sits on exactly one rotation exp(-i a P/2);
  * ``grad_fd``          -- central differences [E(theta_p + h) - E(theta_p - h)] / (2h).
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from .build import build as _build

_lib = None


class _Gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("q0", ctypes.c_int32), ("q1", ctypes.c_int32),
                ("param", ctypes.c_int32), ("angle", ctypes.c_double)]


def lib():
    global _lib
    if _lib is None:
        path = _build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        gp = ctypes.POINTER(_Gate)
        L.orc_run.argtypes = [ctypes.c_int, gp, ctypes.c_int, dp, dp]
        L.orc_run.restype = None
        L.orc_pauli_expectation.argtypes = [ctypes.c_int, dp, ctypes.c_int, ip, ctypes.c_char_p]
        L.orc_pauli_expectation.restype = ctypes.c_double
        L.orc_energy.argtypes = [ctypes.c_int, gp, ctypes.c_int, dp, ctypes.c_int, dp, ip, ip,
                                 ctypes.c_char_p, dp]
        L.orc_energy.restype = ctypes.c_double
        L.orc_grad_adjoint.argtypes = [ctypes.c_int, gp, ctypes.c_int, dp, ctypes.c_int,
                                       ctypes.c_int, dp, ip, ip, ctypes.c_char_p, dp, dp]
        L.orc_grad_adjoint.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _gates(gates):
    arr = (_Gate * max(1, len(gates)))()
    for i, (k, q0, q1, p, a) in enumerate(gates):
        arr[i] = _Gate(int(k), int(q0), int(q1), int(p), float(a))
    return arr


def _terms(terms):
    coeff = np.array([float(c) for c, _, _ in terms], dtype=np.float64)
    off = np.zeros(len(terms) + 1, dtype=np.int32)
    sites, letters = [], []
    for t, (_, s, l) in enumerate(terms):
        if len(s) != len(l):
            raise ValueError("each site needs exactly one Pauli letter")
        sites.extend(int(x) for x in s)
        letters.append(l)
        off[t + 1] = off[t] + len(s)
    sites = np.array(sites if sites else [0], dtype=np.int32)
    return coeff, off, sites, "".join(letters).encode()


def _theta(theta, n_params):
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(-1))
    if th.size < max(1, n_params):
        th = np.concatenate([th, np.zeros(max(1, n_params) - th.size)])
    return th


def statevector(n, gates, theta):
    """Return U(theta)|0...0> as a complex128 vector of length 2^n."""
    psi = np.zeros(2 ** n, dtype=np.complex128)
    th = _theta(theta, 1 + max([g[3] for g in gates] + [0]))
    lib().orc_run(n, _gates(gates), len(gates), _dp(th), _dp(psi.view(np.float64)))
    return psi


def pauli_expectation(n, psi, sites, letters):
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    s = np.array(sites, dtype=np.int32)
    return lib().orc_pauli_expectation(n, _dp(psi.view(np.float64)), len(sites), _ip(s),
                                       letters.encode())


def energy_terms(n, gates, terms, theta):
    """Per-term expectation values <psi|P_t|psi> and the energy sum_t c_t <P_t>."""
    coeff, off, sites, letters = _terms(terms)
    th = _theta(theta, 1 + max([g[3] for g in gates] + [0]))
    et = np.zeros(len(terms), dtype=np.float64)
    E = lib().orc_energy(n, _gates(gates), len(gates), _dp(th), len(terms), _dp(coeff), _ip(off),
                         _ip(sites), letters, _dp(et))
    return E, et


def energy(n, gates, terms, theta):
    return energy_terms(n, gates, terms, theta)[0]


def grad_adjoint(n, gates, terms, theta, n_params):
    """(E, dE/dtheta) from the C oracle's own adjoint sweep."""
    coeff, off, sites, letters = _terms(terms)
    th = _theta(theta, n_params)
    g = np.zeros(max(1, n_params), dtype=np.float64)
    E = np.zeros(1, dtype=np.float64)
    rc = lib().orc_grad_adjoint(n, _gates(gates), len(gates), _dp(th), n_params, len(terms),
                                _dp(coeff), _ip(off), _ip(sites), letters, _dp(E), _dp(g))
    if rc != 0:
        raise MemoryError("oracle adjoint: allocation failed")
    return float(E[0]), g[:n_params].copy()


def grad_param_shift(n, gates, terms, theta, params):
    """Parameter-shift rule for each index in ``params`` (one rotation per parameter)."""
    th = np.array(theta, dtype=np.float64).reshape(-1)
    out = np.zeros(len(params))
    for i, p in enumerate(params):
        tp, tm = th.copy(), th.copy()
        tp[p] += math.pi / 2
        tm[p] -= math.pi / 2
        out[i] = 0.5 * (energy(n, gates, terms, tp) - energy(n, gates, terms, tm))
    return out


def grad_fd(n, gates, terms, theta, params, h=1e-3):
    """Central finite differences with step ``h``."""
    th = np.array(theta, dtype=np.float64).reshape(-1)
    out = np.zeros(len(params))
    for i, p in enumerate(params):
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        out[i] = (energy(n, gates, terms, tp) - energy(n, gates, terms, tm)) / (2 * h)
    return out


def omp_threads() -> int:
    """Threads the OpenMP runtime will use (OMP_NUM_THREADS, else the affinity set)."""
    env = os.environ.get("OMP_NUM_THREADS")
    if env:
        return int(env)
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1
