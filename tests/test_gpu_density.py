"""GPU parity of the partial trace (reduced density operators) against the CPU oracle."""
import math

import numpy as np
import pytest

from oracle import dense, density
from paper_2112_10239_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _tol(rho_ref):
    # FP32 state and sums: entries within 1e-5 of the largest entry (|rho_ij| <= 1)
    return 1e-5 * max(1.0, float(np.max(np.abs(rho_ref))))


def _random_state(n, seed):
    rng = np.random.default_rng(seed)
    psi = rng.normal(size=2 ** n) + 1j * rng.normal(size=2 ** n)
    return psi / np.linalg.norm(psi)


def _trace_dev(tlq, psi, n, keep):
    import torch
    from paper_2112_10239_gb300 import binding as B
    p = torch.tensor(np.ascontiguousarray(psi.astype(np.complex64)).view(np.float32), device="cuda")
    m = len(keep)
    r = torch.empty(2 * 4 ** m, dtype=torch.float32, device="cuda")
    B.tlq_partial_trace_dev(tlq.h, p.data_ptr(), n, keep, r.data_ptr(), None)
    torch.cuda.synchronize()
    return r.cpu().numpy().view(np.complex64).reshape(2 ** m, 2 ** m).astype(np.complex128)


@pytest.mark.parametrize("n,keep", [(1, [0]), (2, [1]), (3, [0, 2]), (6, [5, 1, 3]), (9, list(range(9))),
                                    (10, [0, 1, 2, 3, 4]), (12, [11, 3, 7, 0, 5, 9, 2]), (14, [2, 4, 6, 8, 10, 12, 13]),
                                    (16, [0]), (20, [19, 18]), (13, list(range(13))),
                                    (16, [15, 0, 2, 3, 5, 6, 8, 9, 11, 12, 13, 14]), (15, list(range(3, 15)))])
def test_partial_trace_random_states(tlq, n, keep):
    # ragged and degenerate shapes: m = n (pure rho), m = 1 with long k (split k range),
    # scattered kept qubits, outputs smaller than one 64 x 64 tile and spanning many tiles;
    # m = 12 with k = 16 and k = 8 (one chunk per tile) run the persistent warp-specialised
    # kernel (528 tiles of 128 x 128)
    psi = _random_state(n, seed=n * 31 + len(keep))
    rho = _trace_dev(tlq, psi, n, keep)
    ref = density.reduced_density(psi.astype(np.complex64).astype(np.complex128), n, keep)
    assert np.max(np.abs(rho - ref)) <= _tol(ref)
    assert np.max(np.abs(rho - rho.conj().T)) == 0.0   # written as exact mirrors


def test_partial_trace_paper_shapes_sampled(tlq):
    # n = 20 to m = 14 and m = 10 (the paper's partial-trace sizes); m = 14 sampled
    n = 20
    psi = _random_state(n, seed=7)
    psi32 = psi.astype(np.complex64).astype(np.complex128)
    rng = np.random.default_rng(3)
    keep14 = sorted(int(q) for q in rng.choice(n, 14, replace=False))
    rho = _trace_dev(tlq, psi, n, keep14)
    P = density.split_matrix(psi32, n, keep14)
    for _ in range(200):
        i, j = (int(x) for x in rng.integers(0, 2 ** 14, 2))
        want = np.dot(P[i], P[j].conj())
        assert abs(rho[i, j] - want) <= 1e-5 * max(1e-6, abs(want)) + 1e-9
    assert abs(np.trace(rho) - 1) < 1e-4
    keep10 = list(range(5, 15))
    rho10 = _trace_dev(tlq, psi, n, keep10)
    ref10 = density.reduced_density(psi32, n, keep10)
    assert np.max(np.abs(rho10 - ref10)) <= _tol(ref10)


def test_partial_trace_deterministic(tlq):
    psi = _random_state(18, seed=1)
    a = _trace_dev(tlq, psi, 18, [0, 1, 2])
    b = _trace_dev(tlq, psi, 18, [0, 1, 2])
    assert np.array_equal(a, b)


def test_reduced_density_of_circuits(tlq):
    from paper_2112_10239_gb300 import binding as B
    for prob, keep in ((W.qaoa_problem(12, 2, 1, seed=3), [0, 5, 11]),
                       (W.random_nonlocal_problem(9, 2, 1, seed=2), [8, 1]),
                       (W.tfim_problem(10, 3, 1, seed=4), [4, 5, 6])):
        c, h = tlq.problem(prob)
        try:
            rho = B.tlq_reduced_density(tlq.h, c.h, prob.theta[0], keep)
        finally:
            c.close()
            h.close()
        psi = dense.statevector(prob.n, prob.gates, prob.theta[0])
        ref = density.reduced_density(psi, prob.n, keep)
        assert np.max(np.abs(rho - ref)) <= _tol(ref)


def test_reduced_density_light_cone_window_n500(tlq):
    # n = 500, L = 4 brick-wall: rho of three middle qubits from the window of their backward
    # light cone equals the oracle's on its own padded window (exact by causality)
    from oracle import windows
    from paper_2112_10239_gb300 import binding as B
    prob = W.tfim_problem(500, 4, 1, seed=6)
    keep = [250, 251, 253]
    c, h = tlq.problem(prob)
    try:
        rho = B.tlq_reduced_density(tlq.h, c.h, prob.theta[0], keep)
    finally:
        c.close()
        h.close()
    qubits, kept = windows.cone(prob.gates, keep)
    lo, hi = min(qubits), max(qubits)
    sub = [(k, q0 - lo, (q1 - lo) if q1 >= 0 else -1, p, a)
           for (k, q0, q1, p, a) in (prob.gates[g] for g in sorted(kept))]
    psi = dense.statevector(hi - lo + 1, sub, prob.theta[0])
    ref = density.reduced_density(psi, hi - lo + 1, [q - lo for q in keep])
    assert np.max(np.abs(rho - ref)) <= _tol(ref)
    assert abs(np.trace(rho).real - 1) < 1e-5
