"""GPU parity of the small-circuit energy kernel (n <= 10, energies only) against the oracle.

Energy-only calls on circuits of at most ten qubits run one CTA per parameter set with the
whole state in shared memory; these tests check them against the complex128 oracle on local
and non-local circuits, fixed angles, multi-site Pauli strings and batches, and against the
energy the gradient call (cone or dense path) returns for the same circuits.
"""
import math

import numpy as np
import pytest

from oracle import dense
from paper_2112_10239_gb300 import workloads as W
from parity import check_energy

pytestmark = pytest.mark.gpu


def _energies(tlq, prob):
    from paper_2112_10239_gb300 import binding as B
    c, h = tlq.problem(prob)
    try:
        E = B.tlq_expectation(tlq.h, c.h, h.h, prob.theta)
        Eg, _ = B.tlq_expectation_grad(tlq.h, c.h, h.h, prob.theta)
        return E, Eg
    finally:
        c.close()
        h.close()


def _oracle(prob):
    return np.array([dense.energy(prob.n, prob.gates, prob.terms, th) for th in prob.theta])


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 10])
def test_tiny_local_circuits(tlq, n):
    # mixed RX/RY, RZ on random qubits, CZ / RZZ on random neighbours, X/Y/Z one- and two-site
    # terms, three parameter sets
    prob = W.random_local_problem(n, 3, 3, seed=200 + n)
    E, Eg = _energies(tlq, prob)
    Er = _oracle(prob)
    check_energy(E, Er)
    check_energy(Eg, Er)


@pytest.mark.parametrize("n", [4, 7, 10])
def test_tiny_nonlocal_circuits(tlq, n):
    # two-qubit gates between arbitrary qubits, shared and fixed angles, strings of 1-3 sites
    prob = W.random_nonlocal_problem(n, 3, 2, seed=300 + n)
    E, Eg = _energies(tlq, prob)
    Er = _oracle(prob)
    check_energy(E, Er)
    check_energy(Eg, Er)


def test_tiny_tfim_n8_and_closed_forms(tlq):
    from paper_2112_10239_gb300 import binding as B
    prob = W.tfim_n8_L2()
    E, _ = _energies(tlq, prob)
    check_energy(E, _oracle(prob))
    # GHZ construction with fixed angles: <Z0 Z5> = 1, <X^6> = (-1)^5
    half = math.pi / 2
    n = 6
    gates = [(W.RY, 0, -1, -1, half)]
    for t in range(1, n):
        gates += [(W.RY, t, -1, -1, half), (W.CZ, t - 1, t, -1, 0.0), (W.RY, t, -1, -1, -half)]
    terms = [(1.0, (0, n - 1), "ZZ"), (0.5, tuple(range(n)), "X" * n)]
    ghz = W.Problem(n=n, gates=gates, n_params=0, terms=terms, theta=np.zeros((1, 0)))
    c, h = tlq.problem(ghz)
    try:
        Eghz = B.tlq_expectation(tlq.h, c.h, h.h, ghz.theta)
    finally:
        c.close()
        h.close()
    assert abs(Eghz[0] - (1.0 - 0.5)) < 1e-5
