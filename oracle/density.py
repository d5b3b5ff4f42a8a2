"""Reduced density operators of pure states: the plain definition of the partial trace.

Test infrastructure only (see the package docstring): never imported by the product path.

TensorLy-Quantum (Sec. 2 and Sec. 3, Fig. 1 left) offers partial traces of density
operators and times the full-rank partial trace of an n = 20 qubit system down to m = 14
and m = 10 qubits. For a pure state |psi> the density operator is rho = |psi><psi|, and
tracing out the qubits B outside the kept set A gives

    rho_A[i, j] = sum_k psi(i, k) conj(psi(j, k)),

where psi(i, k) is the amplitude whose kept qubits take the bit pattern i and whose traced
qubits take the pattern k. Index convention (the same as for states): bit q of a state
index is qubit q; bit t of i is qubit keep[t] for the keep list sorted ascending, and bit u
of k is the u-th lowest traced qubit. The routine below writes that sum out with numpy
(a reshape, a transpose and one matrix product); nothing is blocked or reordered.
"""
from __future__ import annotations

import numpy as np


def split_matrix(psi, n, keep):
    """Psi[i, k] = psi(i, k) as a 2^m x 2^(n-m) complex128 matrix (keep sorted ascending)."""
    keep = sorted(int(q) for q in keep)
    if len(set(keep)) != len(keep) or any(q < 0 or q >= n for q in keep):
        raise ValueError("keep must list distinct qubits in [0, n)")
    traced = [q for q in range(n) if q not in keep]
    # numpy's C order puts qubit n-1 on axis 0; axis a holds qubit n-1-a
    t = np.asarray(psi, dtype=np.complex128).reshape((2,) * n)
    order = [n - 1 - q for q in reversed(keep)] + [n - 1 - q for q in reversed(traced)]
    return t.transpose(order).reshape(2 ** len(keep), 2 ** len(traced))


def reduced_density(psi, n, keep):
    """rho_A = Tr_B |psi><psi| as a 2^m x 2^m complex128 matrix (keep sorted ascending)."""
    P = split_matrix(psi, n, keep)
    return P @ P.conj().T
