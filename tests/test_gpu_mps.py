"""GPU parity of the exact MPS route (tlq_mps_expectation_grad[_dev]) against the CPU oracle.

The route builds the circuit's exact matrix-product state (bond dimension 2^gates per pair),
sweeps left and right environments and reads energies and the full gradient per site. The
oracle is the plain statevector definition with its own adjoint (oracle/dense.py) and, at n=500,
the padded light-cone windows (oracle/windows.py).
"""
import math

import numpy as np
import pytest

from oracle import dense, windows
from paper_2112_10239_gb300 import workloads as W
from parity import check_energy, check_grad

pytestmark = pytest.mark.gpu


def _mps(tlq, prob, prec=0, grad=True, theta=None, terms=None):
    from paper_2112_10239_gb300 import binding as B
    p = prob if terms is None else W.Problem(prob.n, prob.gates, prob.n_params, terms, prob.theta)
    c, h = tlq.problem(p)
    try:
        return B.tlq_mps_expectation(tlq.h, c.h, h.h, p.theta if theta is None else theta, prec, grad)
    finally:
        c.close()
        h.close()


def _oracle(prob, terms=None, theta=None):
    terms = prob.terms if terms is None else terms
    th = prob.theta if theta is None else theta
    out = [dense.grad_adjoint(prob.n, prob.gates, terms, t, prob.n_params) for t in th]
    return np.array([e for e, _ in out]), np.array([g for _, g in out])


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("prec", [0, 2])
def test_random_chain_circuits(tlq, seed, prec):
    # RX/RY per qubit, RZ on a random subset, CZ / RZZ on random neighbouring pairs (bond
    # dimensions differ from pair to pair), X/Y/Z one- and two-site terms plus strings over
    # non-adjacent sites (identity inside the span), three parameter sets
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(2, 13))
    L = int(rng.integers(1, 5))
    prob = W.random_local_problem(n, L, 3, seed=800 + seed)
    terms = list(prob.terms)
    if n > 2:
        terms += [(0.37, (0, n - 1), "XY"), (-0.21, (n - 1, 1, 0), "ZXY")]
    E, g = _mps(tlq, prob, prec, terms=terms)
    Er, gr = _oracle(prob, terms)
    check_energy(E, Er, prec)
    check_grad(g, gr, prec)
    Ee, _ = _mps(tlq, prob, prec, grad=False, terms=terms)
    check_energy(Ee, Er, prec)


@pytest.mark.parametrize("n,L,prec", [(1, 3, 0), (2, 1, 2), (10, 5, 2), (12, 6, 0), (20, 6, 0)])
def test_tfim_bond_dimensions(tlq, n, L, prec):
    # bond dimension 2^L up to 64 (FP32) and 32 (FP64): the widest use several shared-memory
    # passes per site; n=20, L=6 is the 64-set benchmark circuit (four sets here)
    prob = W.tfim_problem(n, L, 4 if n == 20 else 2, seed=n + 31 * L, h_range=(0.5, 1.5))
    E, g = _mps(tlq, prob, prec)
    Er, gr = _oracle(prob)
    check_energy(E, Er, prec)
    check_grad(g, gr, prec)


def test_agrees_with_cone_path_and_batch_invariant(tlq):
    # the same circuit through the causal-cone kernels; one set alone equals itself in a batch
    from paper_2112_10239_gb300 import binding as B
    prob = W.tfim_problem(16, 4, 8, seed=12, h_range=(0.5, 1.5))
    E, g = _mps(tlq, prob)
    c, h = tlq.problem(prob)
    try:
        Ec, gc = B.tlq_expectation_grad(tlq.h, c.h, h.h, prob.theta)
    finally:
        c.close()
        h.close()
    check_energy(E, Ec)
    check_grad(g, gc)
    E1, g1 = _mps(tlq, prob, theta=prob.theta[5:6])
    assert E1[0] == E[5] and np.array_equal(g1[0], g[5])


def test_device_pointer_call_matches_host_call(tlq):
    import torch
    from paper_2112_10239_gb300 import binding as B
    prob = W.tfim_problem(12, 3, 5, seed=4, h_range=(0.5, 1.5))
    E, g = _mps(tlq, prob)
    c, h = tlq.problem(prob)
    try:
        th = torch.tensor(prob.theta, dtype=torch.float64, device="cuda")
        Ed = torch.empty(5, dtype=torch.float64, device="cuda")
        Gd = torch.empty(prob.theta.shape, dtype=torch.float64, device="cuda")
        s = torch.cuda.current_stream()
        B.tlq_mps_expectation_grad_dev(tlq.h, c.h, h.h, th.data_ptr(), 5, B.TLQ_FP32, Ed.data_ptr(), Gd.data_ptr(),
                                       s.cuda_stream)
        torch.cuda.synchronize()
    finally:
        c.close()
        h.close()
    assert np.array_equal(Ed.cpu().numpy(), E) and np.array_equal(Gd.cpu().numpy(), g)


def test_fixed_angles_ghz_closed_form(tlq):
    # GHZ ladder with fixed angles: <Z0 Z5> = 1, <X^6> = (-1)^5, <Y1 Y2> = 0
    half = math.pi / 2
    n = 6
    gates = [(W.RY, 0, -1, -1, half)]
    for t in range(1, n):
        gates += [(W.RY, t, -1, -1, half), (W.CZ, t - 1, t, -1, 0.0), (W.RY, t, -1, -1, -half)]
    terms = [(1.0, (0, n - 1), "ZZ"), (0.5, tuple(range(n)), "X" * n), (0.25, (1, 2), "YY")]
    prob = W.Problem(n=n, gates=gates, n_params=0, terms=terms, theta=np.zeros((1, 0)))
    E, _ = _mps(tlq, prob, grad=False)
    assert abs(E[0] - (1.0 - 0.5)) < 1e-5


def test_tfim_n500_L4_B256_sampled(tlq):
    # the n=500 batch (999 terms, 4000 angles, bond dimension 16) on the MPS route; the oracle's
    # padded windows check three sets exactly, and the cone path's result the rest
    from paper_2112_10239_gb300 import binding as B
    prob = W.tfim_n500_L4_B256()
    E, g = _mps(tlq, prob)
    assert E.shape == (256,) and g.shape == (256, 4000)
    cc = windows.ConeCache(prob.gates, prob.terms)
    for b in (0, 255):
        check_energy(E[b:b + 1], [cc.energy(prob.theta[b])])
    Er, gr = cc.grad(prob.theta[77], prob.n_params)
    check_energy(E[77:78], [Er])
    check_grad(g[77], gr)
    c, h = tlq.problem(prob)
    try:
        Ec, gc = B.tlq_expectation_grad(tlq.h, c.h, h.h, prob.theta)
    finally:
        c.close()
        h.close()
    check_energy(E, Ec)
    check_grad(g, gc)


def test_unsupported_circuits(tlq):
    from paper_2112_10239_gb300 import binding as B
    q = W.qaoa_problem(10, 2, 1, seed=0)
    with pytest.raises(B.TLQError) as ei:
        _mps(tlq, q)
    assert ei.value.status == B.TLQ_EUNSUPPORTED
    # bond dimension 64 runs in FP32 only
    p = W.tfim_problem(8, 6, 1, seed=2)
    with pytest.raises(B.TLQError) as ei:
        _mps(tlq, p, prec=2)
    assert ei.value.status == B.TLQ_EUNSUPPORTED
