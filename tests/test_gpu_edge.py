"""Degenerate and boundary inputs through the C-ABI, against closed forms or the CPU oracle:
an empty circuit, parameters no gate uses, circuits with fixed angles only, terms with zero
coefficients, qubits without gates, and a large batch of parameter sets."""
import math

import numpy as np
import pytest

from oracle import dense
from paper_2112_10239_gb300 import workloads as W
from parity import check_energy, check_grad

pytestmark = pytest.mark.gpu


def _run(tlq, prob, theta, prec=0, grad=True):
    from paper_2112_10239_gb300 import binding as B
    c, h = tlq.problem(prob)
    try:
        if grad:
            return B.tlq_expectation_grad(tlq.h, c.h, h.h, theta, prec)
        return B.tlq_expectation(tlq.h, c.h, h.h, theta, prec), None
    finally:
        c.close()
        h.close()


def _oracle(prob, theta):
    out = [dense.grad_adjoint(prob.n, prob.gates, prob.terms, th, prob.n_params) for th in theta]
    return np.array([e for e, _ in out]), np.array([g for _, g in out])


@pytest.mark.parametrize("n", [3, 20, 60])
@pytest.mark.parametrize("prec", [0, 2])
def test_empty_circuit_closed_form(tlq, n, prec):
    # no gates: the state is |0..0>, so <P> = 1 for Z-only strings and 0 for any X/Y letter;
    # with parameters declared but unused every gradient entry is exactly zero
    rng = np.random.default_rng(n)
    terms = []
    for _ in range(2 * n):
        k = int(rng.integers(1, 3))
        q = int(rng.integers(0, n - k + 1))
        sites = tuple(range(q, q + k))
        terms.append((float(rng.uniform(-1, 1)), sites, "".join("XYZ"[int(rng.integers(3))] for _ in sites)))
    prob = W.Problem(n=n, gates=[], n_params=4, terms=terms, theta=rng.uniform(0, 6, size=(3, 4)))
    want = sum(c for c, _, l in terms if set(l) <= {"Z"})
    E, G = _run(tlq, prob, prob.theta, prec)
    check_energy(E, [want] * 3, prec)
    assert np.all(G == 0.0)


@pytest.mark.parametrize("prec", [0, 2])
def test_unused_parameters_have_zero_gradient(tlq, prec):
    # the brick-wall ansatz with 2 extra parameters no gate carries
    base = W.tfim_problem(10, 3, 2, seed=3, h_range=(0.5, 1.5))
    P = base.n_params + 2
    theta = np.concatenate([base.theta, np.full((2, 2), 0.7)], axis=1)
    prob = W.Problem(n=base.n, gates=base.gates, n_params=P, terms=base.terms, theta=theta)
    E, G = _run(tlq, prob, theta, prec)
    Er, gr = _oracle(prob, theta)
    check_energy(E, Er, prec)
    check_grad(G, gr, prec)
    assert np.all(G[:, -2:] == 0.0)


@pytest.mark.parametrize("nonlocal_", [False, True])
def test_fixed_angles_only(tlq, nonlocal_):
    # every gate has a fixed angle (n_params = 0): the energy against the oracle, on the cone path
    # and on the dense path (a two-qubit gate between distant qubits)
    rng = np.random.default_rng(11 if nonlocal_ else 12)
    n = 14
    gates = []
    for _ in range(3):
        for q in range(n):
            gates.append((W.RY if rng.random() < 0.5 else W.RX, q, -1, -1, float(rng.uniform(0, 6))))
        for q in range(0, n - 1, 2):
            gates.append((W.RZZ, q, q + 1, -1, float(rng.uniform(0, 6))))
    if nonlocal_:
        gates.append((W.CZ, 0, n - 1, -1, 0.0))
    terms = [(1.0, (i, i + 1), "ZZ") for i in range(n - 1)] + [(0.5, (i,), "X") for i in range(n)]
    prob = W.Problem(n=n, gates=gates, n_params=0, terms=terms, theta=np.zeros((2, 0)))
    E, G = _run(tlq, prob, prob.theta)
    want = dense.energy(n, gates, terms, np.zeros(0))
    check_energy(E, [want, want])
    assert G.shape == (2, 0)


def test_zero_coefficients_and_idle_qubits(tlq):
    # terms with coefficient 0 contribute nothing; qubits 5..7 carry no gate at all
    n = 12
    gates, P = [], 0
    for _ in range(2):
        for q in range(n):
            if 5 <= q <= 7:
                continue
            gates.append((W.RY, q, -1, P, 0.0)); P += 1
        for q in range(0, 4):
            gates.append((W.CZ, q, q + 1, -1, 0.0))
        for q in range(8, n - 1):
            gates.append((W.RZZ, q, q + 1, P, 0.0)); P += 1
    terms = [(0.0, (i, i + 1), "ZZ") for i in range(n - 1)] + [(0.8 if i % 3 else 0.0, (i,), "X") for i in range(n)]
    terms += [(1.3, (6,), "Z"), (0.0, (2, 9), "YY")]
    theta = np.random.default_rng(5).uniform(0, 6, size=(3, P))
    prob = W.Problem(n=n, gates=gates, n_params=P, terms=terms, theta=theta)
    E, G = _run(tlq, prob, theta)
    Er, gr = _oracle(prob, theta)
    check_energy(E, Er)
    check_grad(G, gr)


def test_large_batch_sampled(tlq):
    # 2048 parameter sets in one call; sampled sets against the oracle, and the batch agrees bit
    # for bit with the same sets evaluated in a small batch
    prob = W.tfim_problem(12, 3, 2048, seed=17, h_range=(0.5, 1.5))
    E, G = _run(tlq, prob, prob.theta)
    idx = [0, 1, 777, 1500, 2047]
    Er, gr = _oracle(prob, prob.theta[idx])
    check_energy(E[idx], Er)
    check_grad(G[idx], gr)
    Es, Gs = _run(tlq, prob, prob.theta[idx])
    assert np.array_equal(Es, E[idx]) and np.array_equal(Gs, G[idx])
