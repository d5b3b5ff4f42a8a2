"""GPU parity of the dense statevector path (through the C-ABI) against the CPU oracle."""
import math

import numpy as np
import pytest

from oracle import dense
from paper_2112_10239_gb300 import workloads as W
from parity import check_energy, check_grad

pytestmark = pytest.mark.gpu


def _energy(ctx, prob, theta=None):
    from paper_2112_10239_gb300 import binding as B
    c, h = ctx.problem(prob)
    try:
        path, *_ = B.tlq_plan_info(ctx.h, c.h, h.h, len(prob.terms))
        E = B.tlq_expectation(ctx.h, c.h, h.h, prob.theta if theta is None else theta)
        return E, path
    finally:
        c.close()
        h.close()


def _oracle(prob, theta):
    return np.array([dense.energy(prob.n, prob.gates, prob.terms, th) for th in theta])


@pytest.fixture(scope="module")
def plain_ctx():
    """A context whose fuse_k = 1 selects plain per-gate sweeps (the baseline path)."""
    from paper_2112_10239_gb300 import binding as B
    cfg = B.tlq_config(0, 0, 0, B.TLQ_FP32, 1)
    import ctypes
    h = ctypes.c_void_p()
    B._check(B.lib().tlq_init(ctypes.byref(cfg), ctypes.byref(h)))
    ctx = B.Context.__new__(B.Context)
    ctx.h = h
    yield ctx
    ctx.close()


@pytest.mark.parametrize("n,p,seed", [(10, 1, 0), (12, 2, 1), (14, 3, 2), (16, 4, 3), (20, 4, 4)])
def test_qaoa_reduced_vs_oracle(tlq, n, p, seed):
    from paper_2112_10239_gb300 import binding as B
    prob = W.qaoa_problem(n, p, 3, seed)
    E, path = _energy(tlq, prob)
    assert path == B.TLQ_PATH_DENSE
    check_energy(E, _oracle(prob, prob.theta))


def test_qaoa_n24_vs_oracle(tlq):
    prob = W.qaoa_problem(24, 4, 1, seed=7)
    E, _ = _energy(tlq, prob)
    check_energy(E, _oracle(prob, prob.theta))


def test_qaoa_n28_closed_forms(tlq):
    # full size: p=1 from |0..0> gives E = |edges| cos^2(beta_1); every beta = 0 gives E = |edges|
    prob = W.qaoa_n28_p4(B=2)
    m = len(prob.meta["edges"])
    assert m == 42
    E, _ = _energy(tlq, prob)
    assert np.all(np.abs(E) <= m + 1e-4)
    th = prob.theta.copy()
    th[:, 1::2] = 0.0
    E0, _ = _energy(tlq, prob, th)
    check_energy(E0, [m, m])
    one = W.qaoa_problem(28, 1, 3, seed=2, edges=prob.meta["edges"])
    E1, _ = _energy(tlq, one)
    check_energy(E1, [m * math.cos(b) ** 2 for b in one.theta[:, 1]])


def test_qaoa_n28_deterministic(tlq):
    prob = W.qaoa_n28_p4()
    a, _ = _energy(tlq, prob)
    b, _ = _energy(tlq, prob)
    assert a[0] == b[0]


@pytest.mark.parametrize("seed", range(4))
def test_nonlocal_mixed_circuits(tlq, seed):
    # non-adjacent RZZ/CZ, RX/RY/RZ with distinct angles, X/Y/Z terms of 1-3 sites
    rng = np.random.default_rng(50 + seed)
    n = int(rng.integers(4, 15))
    gates, P = [], 0
    for _ in range(3):
        for q in range(n):
            gates.append((W.RY if rng.random() < 0.5 else W.RX, q, -1, P, 0.0)); P += 1
        for q in range(n):
            if rng.random() < 0.5:
                gates.append((W.RZ, q, -1, P, 0.0)); P += 1
        for _ in range(n):
            u, v = rng.choice(n, 2, replace=False)
            if rng.random() < 0.5:
                gates.append((W.CZ, int(u), int(v), -1, 0.0))
            else:
                gates.append((W.RZZ, int(u), int(v), P, 0.0)); P += 1
    terms = []
    for _ in range(2 * n):
        k = int(rng.integers(1, 4))
        sites = tuple(int(s) for s in rng.choice(n, k, replace=False))
        terms.append((float(rng.uniform(-1, 1)), sites, "".join("XYZ"[int(rng.integers(3))] for _ in sites)))
    theta = rng.uniform(0, 2 * math.pi, size=(2, P))
    prob = W.Problem(n=n, gates=gates, n_params=P, terms=terms, theta=theta)
    E, _ = _energy(tlq, prob)
    check_energy(E, _oracle(prob, theta))


@pytest.mark.parametrize("n", [1, 2, 3])
def test_tiny_dense(tlq, n):
    gates = [(W.RY, q, -1, q, 0.0) for q in range(n)]
    if n >= 3:
        gates.append((W.RZZ, 0, 2, n, 0.0))
    P = n + (1 if n >= 3 else 0)
    terms = [(1.0, (0,), "X")] + ([(0.5, (0, n - 1), "ZZ")] if n > 1 else [])
    theta = np.random.default_rng(n).uniform(0, 6, size=(1, P))
    prob = W.Problem(n=n, gates=gates, n_params=P, terms=terms, theta=theta)
    E, _ = _energy(tlq, prob)
    check_energy(E, _oracle(prob, theta))


def test_plain_per_gate_baseline(plain_ctx, tlq):
    # the per-gate sweep baseline agrees with the fused passes and the oracle
    prob = W.qaoa_problem(16, 3, 2, seed=11)
    Ep, _ = _energy(plain_ctx, prob)
    Ef, _ = _energy(tlq, prob)
    Er = _oracle(prob, prob.theta)
    check_energy(Ep, Er)
    check_energy(Ef, Er)
    t = W.tfim_problem(12, 3, 2, seed=1, h_range=(0.5, 1.5))   # cone-path circuit run as plain sweeps
    Ept, _ = _energy(plain_ctx, t)
    check_energy(Ept, _oracle(t, t.theta))


def _grad(ctx, prob, theta=None):
    from paper_2112_10239_gb300 import binding as B
    c, h = ctx.problem(prob)
    try:
        return B.tlq_expectation_grad(ctx.h, c.h, h.h, prob.theta if theta is None else theta)
    finally:
        c.close()
        h.close()


def _oracle_grad(prob, theta):
    out = [dense.grad_adjoint(prob.n, prob.gates, prob.terms, th, prob.n_params) for th in theta]
    return np.array([e for e, _ in out]), np.array([g for _, g in out])


@pytest.mark.parametrize("n,p,seed", [(10, 1, 0), (12, 2, 1), (14, 3, 2), (16, 4, 3), (18, 4, 5)])
def test_qaoa_gradient_vs_oracle(tlq, n, p, seed):
    prob = W.qaoa_problem(n, p, 2, seed)
    E, g = _grad(tlq, prob)
    Er, gr = _oracle_grad(prob, prob.theta)
    check_energy(E, Er)
    check_grad(g, gr)
    # the energy of the gradient call equals the energy-only call (bit for bit on the dense
    # path; up to rounding below 11 qubits, where energy-only calls run the small-circuit kernel)
    E2, _ = _energy(tlq, prob)
    if n > 10:
        assert np.array_equal(E, E2)
    else:
        check_energy(E2, E)


def test_qaoa_n24_gradient_vs_oracle(tlq):
    prob = W.qaoa_problem(24, 4, 1, seed=7)
    E, g = _grad(tlq, prob)
    Er, gr = _oracle_grad(prob, prob.theta)
    check_energy(E, Er)
    check_grad(g, gr)


def test_qaoa_n28_gradient_closed_form(tlq):
    # full size, p = 1: E = |edges| cos^2 beta, dE/dgamma = 0, dE/dbeta = -|edges| sin 2 beta
    full = W.qaoa_n28_p4()
    m = len(full.meta["edges"])
    one = W.qaoa_problem(28, 1, 3, seed=2, edges=full.meta["edges"])
    E, g = _grad(tlq, one)
    check_energy(E, [m * math.cos(b) ** 2 for b in one.theta[:, 1]])
    want = np.stack([np.zeros(3), -m * np.sin(2 * one.theta[:, 1])], axis=1)
    check_grad(g, want)


def test_qaoa_n28_p4_gradient_fused_equals_plain(plain_ctx, tlq):
    # full size p = 4: the fused adjoint passes against the plain per-gate adjoint sweeps
    # (two independent kernel paths), and gamma_1 (a global phase on |0..0>) has zero gradient
    prob = W.qaoa_n28_p4()
    E, g = _grad(tlq, prob)
    Ep, gp = _grad(plain_ctx, prob)
    check_energy(E, Ep)
    check_grad(g, gp)
    assert abs(g[0, 0]) <= 1e-4 * max(1.0, float(np.max(np.abs(g))))


@pytest.mark.parametrize("seed", range(5))
def test_nonlocal_mixed_gradients(tlq, seed):
    # X/Y/Z strings (lam needs the gather kernel), RZ singles, CZ, fixed angles, shared angles
    rng = np.random.default_rng(70 + seed)
    prob = W.random_nonlocal_problem(int(rng.integers(3, 15)), int(rng.integers(1, 4)), 2, 300 + seed)
    E, g = _grad(tlq, prob)
    Er, gr = _oracle_grad(prob, prob.theta)
    check_energy(E, Er)
    check_grad(g, gr)


@pytest.mark.parametrize("n", [14, 19])
def test_diagonal_class_count_forms(tlq, n):
    # Diagonal classes counted both ways in one circuit: classes of at most 64 terms read
    # edge-word tables (the first two per pass), larger ones and the rest loop over distances.
    # RZZ on every pair with one angle (> 64 terms), RZZ on the pairs of the first 11 qubits plus
    # RZ on qubits 0..4 with another (60 terms), three lone RZZ angles and a CZ in the same
    # layer; energy from ZZ on every pair (> 64 terms) plus a small ZZ / Z class and X terms.
    rng = np.random.default_rng(90 + n)
    pairs = [(u, v) for u in range(n) for v in range(u + 1, n)]
    small = [(u, v) for u in range(11) for v in range(u + 1, 11)]
    gates, P = [], 0
    for layer in range(2):
        for q in range(n):
            gates.append((W.RY if (q + layer) % 3 else W.RX, q, -1, P + q, 0.0))
        P += n
        gates += [(W.RZZ, u, v, P, 0.0) for u, v in pairs]
        gates += [(W.RZZ, u, v, P + 1, 0.0) for u, v in small] + [(W.RZ, q, -1, P + 1, 0.0) for q in range(5)]
        for k in range(3):
            gates.append((W.RZZ, k, n - 1 - k, P + 2 + k, 0.0))
        gates.append((W.CZ, 1, n - 2, -1, 0.0))
        P += 5
    for q in range(n):
        gates.append((W.RX, q, -1, P, 0.0))
    P += 1
    terms = [(1.0, (u, v), "ZZ") for u, v in pairs]
    terms += [(0.5, (u, u + 3), "ZZ") for u in range(6)] + [(0.5, (q,), "Z") for q in range(4)]
    terms += [(0.25, (q,), "X") for q in range(0, n, 3)]
    theta = rng.uniform(0, 2 * math.pi, size=(2, P))
    prob = W.Problem(n=n, gates=gates, n_params=P, terms=terms, theta=theta)
    E, g = _grad(tlq, prob)
    Er, gr = _oracle_grad(prob, theta)
    check_energy(E, Er)
    check_grad(g, gr)
    E2, _ = _energy(tlq, prob)
    check_energy(E2, Er)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_tiny_dense_gradient(tlq, n):
    gates = [(W.RY, q, -1, q, 0.0) for q in range(n)] + [(W.RX, q, -1, n + q, 0.0) for q in range(n)]
    P = 2 * n
    if n >= 3:
        gates.append((W.RZZ, 0, 2, P, 0.0))
        gates.append((W.RY, 1, -1, P + 1, 0.0))
        P += 2
    terms = [(1.0, (0,), "X")] + ([(0.5, (0, n - 1), "ZZ"), (-0.25, (n - 1,), "Y")] if n > 1 else [])
    theta = np.random.default_rng(n).uniform(0, 6, size=(2, P))
    prob = W.Problem(n=n, gates=gates, n_params=P, terms=terms, theta=theta)
    E, g = _grad(tlq, prob)
    Er, gr = _oracle_grad(prob, theta)
    check_energy(E, Er)
    check_grad(g, gr)


def test_plain_per_gate_gradient(plain_ctx, tlq):
    for prob in (W.qaoa_problem(14, 3, 2, seed=12), W.random_nonlocal_problem(9, 2, 2, seed=5),
                 W.tfim_problem(10, 3, 2, seed=1, h_range=(0.5, 1.5))):
        E, g = _grad(plain_ctx, prob)
        Er, gr = _oracle_grad(prob, prob.theta)
        check_energy(E, Er)
        check_grad(g, gr)


def test_dense_gradient_deterministic(tlq):
    prob = W.qaoa_problem(20, 4, 2, seed=9)
    a = _grad(tlq, prob)
    b = _grad(tlq, prob)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_dense_fp64_reports_unsupported(tlq):
    from paper_2112_10239_gb300 import binding as B
    prob = W.qaoa_problem(10, 1, 1, seed=0)
    c, h = tlq.problem(prob)
    try:
        with pytest.raises(B.TLQError) as ei:
            B.tlq_expectation_grad(tlq.h, c.h, h.h, prob.theta, B.TLQ_FP64_REF)
        assert ei.value.status == B.TLQ_EUNSUPPORTED
    finally:
        c.close()
        h.close()


def test_dense_largest_state_n31(tlq):
    # n=31, the largest dense state (2^31 complex64 = 16 GiB): QAOA p=1 on a 3-regular graph
    # has the closed form E = |edges| cos^2(beta) from |0..0> (the RZZ layer is a global phase);
    # n=31 is odd, so the graph is built on 30 vertices and qubit 30 stays idle but simulated
    one = W.qaoa_problem(30, 1, 2, seed=4)
    m = len(one.meta["edges"])
    prob = W.Problem(n=31, gates=one.gates, n_params=one.n_params, terms=one.terms, theta=one.theta)
    E, _ = _energy(tlq, prob)
    check_energy(E, [m * math.cos(b) ** 2 for b in one.theta[:, 1]])


def _golden(name):
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)) as f:
        return json.load(f)


@pytest.mark.parametrize("prec", ["fp32", "mixed_tc"])
def test_qaoa_n28_p4_vs_golden_oracle(tlq, prec):
    """Full size, general angles: energy and gradient of the n=28, p=4 QAOA circuit against the
    complex128 oracle's values stored in tests/golden/qaoa_n28_p4.json."""
    from paper_2112_10239_gb300 import binding as B
    g = _golden("qaoa_n28_p4.json")
    gates = [tuple(x) for x in g["gates"]]
    terms = [(c, tuple(s), l) for c, s, l in g["terms"]]
    theta = np.array([g["theta"]], dtype=np.float64)
    c = tlq.circuit(g["n"], gates, g["n_params"])
    h = tlq.hamiltonian(g["n"], terms)
    mode = {"fp32": B.TLQ_FP32, "mixed_tc": B.TLQ_MIXED_TC}[prec]
    try:
        E, G = B.tlq_expectation_grad(tlq.h, c.h, h.h, theta, mode)
        E2 = B.tlq_expectation(tlq.h, c.h, h.h, theta, mode)
    finally:
        c.close()
        h.close()
    check_energy(E, [g["energy"]])
    check_energy(E2, [g["energy"]])
    check_grad(G, np.array([g["grad"]]))


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("prec", ["fp32", "mixed_tc"])
def test_rx_frame_with_xy_terms(tlq, seed, prec):
    """RX-only qubits run in the rotated frame S = diag(1, i) (RX acts as RY there): X/Y letters
    on those qubits are measured as Y / -X. QAOA-style layers (RZZ on random pairs, RX on every
    qubit, RY on a few qubits, so some qubits stay in the plain frame) against random X/Y/Z
    strings of 1-3 sites, energy and gradient against the oracle."""
    from paper_2112_10239_gb300 import binding as B
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(12, 17))
    gates, P = [], 0
    ry_qubits = set(int(q) for q in rng.choice(n, 2, replace=False))
    for _ in range(3):
        for _ in range(n):
            u, v = (int(x) for x in rng.choice(n, 2, replace=False))
            gates.append((W.RZZ, u, v, P, 0.0)); P += 1
        for q in range(n):
            gates.append((W.RY if q in ry_qubits else W.RX, q, -1, P, 0.0)); P += 1
    terms = []
    for _ in range(2 * n):
        k = int(rng.integers(1, 4))
        sites = tuple(int(s) for s in rng.choice(n, k, replace=False))
        terms.append((float(rng.uniform(-1, 1)), sites, "".join("XYZ"[int(rng.integers(3))] for _ in sites)))
    theta = rng.uniform(0, 2 * math.pi, size=(2, P))
    prob = W.Problem(n=n, gates=gates, n_params=P, terms=terms, theta=theta)
    mode = {"fp32": B.TLQ_FP32, "mixed_tc": B.TLQ_MIXED_TC}[prec]
    c, h = tlq.problem(prob)
    try:
        E, G = B.tlq_expectation_grad(tlq.h, c.h, h.h, theta, mode)
        E2 = B.tlq_expectation(tlq.h, c.h, h.h, theta, mode)
    finally:
        c.close()
        h.close()
    Er, gr = _oracle_grad(prob, theta)
    check_energy(E, Er)
    check_energy(E2, Er)
    check_grad(G, gr)
