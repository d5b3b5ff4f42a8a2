"""Exact diagonalisation with an explicit Hamiltonian matrix (n <= 10).

Test infrastructure only (see the package docstring).

TensorLy-Quantum Sec. 3 notes that a matrix-encoded Hamiltonian is infeasible
beyond a few dozen qubits; at n <= 10 it is a 1024 x 1024 matrix and gives an
independent route to <psi|H|psi> and to the variational bound E >= lambda_min(H).
"""
from __future__ import annotations

import numpy as np

_P = {
    "I": np.eye(2, dtype=np.complex128),
    "X": np.array([[0, 1], [1, 0]], dtype=np.complex128),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    "Z": np.array([[1, 0], [0, -1]], dtype=np.complex128),
}


def pauli_matrix(n, sites, letters):
    """Explicit 2^n x 2^n matrix; qubit q is bit q of the index, so the Kronecker
    product runs from qubit n-1 (leftmost factor) down to qubit 0."""
    ops = ["I"] * n
    for s, l in zip(sites, letters):
        ops[s] = l
    M = np.ones((1, 1), dtype=np.complex128)
    for q in range(n - 1, -1, -1):
        M = np.kron(M, _P[ops[q]])
    return M


def hamiltonian_matrix(n, terms):
    if n > 12:
        raise ValueError("explicit Hamiltonians are only built for small n")
    H = np.zeros((2 ** n, 2 ** n), dtype=np.complex128)
    for c, sites, letters in terms:
        H += c * pauli_matrix(n, sites, letters)
    return H


def expectation(H, psi):
    return float(np.real(np.vdot(psi, H @ psi)))


def ground_energy(H):
    return float(np.linalg.eigvalsh(H)[0])
