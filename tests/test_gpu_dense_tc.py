"""GPU parity of the dense statevector path in the mixed-precision tensor-core mode
(TLQ_MIXED_TC: each register group's rotations applied as one 16 x 16 complex block on the
tensor cores, split TF32 products accumulated in FP32) against the CPU oracle, at the same
tolerances as the FP32 path (energy 1e-5 relative, gradient 1e-4)."""
import math

import numpy as np
import pytest

from oracle import dense
from paper_2112_10239_gb300 import workloads as W
from parity import check_energy, check_grad, energy_err, grad_err

pytestmark = pytest.mark.gpu


def _run(ctx, prob, theta=None, grad=False, prec=None):
    from paper_2112_10239_gb300 import binding as B
    prec = B.TLQ_MIXED_TC if prec is None else prec
    th = prob.theta if theta is None else theta
    c, h = ctx.problem(prob)
    try:
        path, *_ = B.tlq_plan_info(ctx.h, c.h, h.h, len(prob.terms))
        assert path == B.TLQ_PATH_DENSE
        if grad:
            return B.tlq_expectation_grad(ctx.h, c.h, h.h, th, prec)
        return B.tlq_expectation(ctx.h, c.h, h.h, th, prec), None
    finally:
        c.close()
        h.close()


def _oracle_energy(prob, theta):
    return np.array([dense.energy(prob.n, prob.gates, prob.terms, th) for th in theta])


def _oracle_grad(prob, theta):
    out = [dense.grad_adjoint(prob.n, prob.gates, prob.terms, th, prob.n_params) for th in theta]
    return np.array([e for e, _ in out]), np.array([g for _, g in out])


@pytest.mark.parametrize("n,p,seed", [(12, 1, 0), (12, 2, 1), (14, 3, 2), (16, 4, 3), (20, 4, 4), (22, 3, 5)])
def test_qaoa_tc_energy_vs_oracle(tlq, n, p, seed):
    prob = W.qaoa_problem(n, p, 3, seed)
    E, _ = _run(tlq, prob)
    check_energy(E, _oracle_energy(prob, prob.theta))


def test_qaoa_n24_tc_vs_oracle(tlq):
    prob = W.qaoa_problem(24, 4, 1, seed=7)
    E, g = _run(tlq, prob, grad=True)
    Er, gr = _oracle_grad(prob, prob.theta)
    check_energy(E, Er)
    check_grad(g, gr)


@pytest.mark.parametrize("seed", range(5))
def test_nonlocal_mixed_tc(tlq, seed):
    # RX and RY mixed within register groups (complex blocks), partial groups, RZ/RZZ/CZ,
    # fixed and shared angles, X/Y/Z strings of 1-3 sites
    rng = np.random.default_rng(90 + seed)
    prob = W.random_nonlocal_problem(int(rng.integers(12, 19)), int(rng.integers(1, 4)), 2, 400 + seed)
    E, g = _run(tlq, prob, grad=True)
    Er, gr = _oracle_grad(prob, prob.theta)
    check_energy(E, Er)
    check_grad(g, gr)
    E2, _ = _run(tlq, prob)
    check_energy(E2, Er)


def test_qaoa_n28_tc_closed_forms(tlq):
    full = W.qaoa_n28_p4(B=2)
    m = len(full.meta["edges"])
    th = full.theta.copy()
    th[:, 1::2] = 0.0
    E0, _ = _run(tlq, full, th)
    check_energy(E0, [m, m])
    one = W.qaoa_problem(28, 1, 3, seed=2, edges=full.meta["edges"])
    E1, _ = _run(tlq, one)
    check_energy(E1, [m * math.cos(b) ** 2 for b in one.theta[:, 1]])


def test_tc_matches_fp32_path(tlq):
    # the two precisions agree at the FP32 contract on a mid-size circuit
    from paper_2112_10239_gb300 import binding as B
    prob = W.qaoa_problem(22, 4, 2, seed=11)
    Et, gt = _run(tlq, prob, grad=True)
    Ef, gf = _run(tlq, prob, grad=True, prec=B.TLQ_FP32)
    assert energy_err(Et, Ef) <= 1e-5 and grad_err(gt, gf) <= 1e-4


def test_tc_deterministic(tlq):
    prob = W.qaoa_problem(20, 3, 1, seed=12)
    a, _ = _run(tlq, prob)
    b, _ = _run(tlq, prob)
    assert a[0] == b[0]
