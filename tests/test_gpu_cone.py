"""GPU parity of the causal-cone path (through the C-ABI) against the CPU oracle."""
import json
import math
import os

import numpy as np
import pytest

from oracle import dense, windows
from paper_2112_10239_gb300 import workloads as W
from parity import check_energy, check_grad

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def _run(tlq, prob, theta=None, prec=0, grad=True):
    from paper_2112_10239_gb300 import binding as B
    c, h = tlq.problem(prob)
    th = prob.theta if theta is None else theta
    try:
        if grad:
            return B.tlq_expectation_grad(tlq.h, c.h, h.h, th, prec)
        return B.tlq_expectation(tlq.h, c.h, h.h, th, prec), None
    finally:
        c.close()
        h.close()


def _oracle(prob, theta, grad=True):
    if grad:
        out = [dense.grad_adjoint(prob.n, prob.gates, prob.terms, th, prob.n_params) for th in theta]
        return np.array([e for e, _ in out]), np.array([g for _, g in out])
    return np.array([dense.energy(prob.n, prob.gates, prob.terms, th) for th in theta]), None


@pytest.mark.parametrize("name", ["tfim_n8_L2.json", "local_mixed_n7_L3.json"])
@pytest.mark.parametrize("prec", [0, 2])
def test_golden_fixtures(tlq, name, prec):
    d = json.load(open(os.path.join(HERE, "golden", name)))
    prob = W.Problem(n=d["n"], gates=[tuple(g) for g in d["gates"]], n_params=d["n_params"],
                     terms=[(c, tuple(s), l) for c, s, l in d["terms"]], theta=np.array([d["theta"]]))
    E, g = _run(tlq, prob, prec=prec)
    check_energy(E, [d["energy"]], prec)
    check_grad(g[0], d["grad"], prec)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("prec", [0, 2])
def test_random_local_circuits(tlq, seed, prec):
    # mixed RX/RY/RZ/RZZ/CZ, X/Y/Z letters, single and two-site terms, ragged batch
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(3, 13))
    L = int(rng.integers(1, 5))
    prob = W.random_local_problem(n, L, 3, seed)
    E, g = _run(tlq, prob, prec=prec)
    Er, gr = _oracle(prob, prob.theta)
    check_energy(E, Er, prec)
    check_grad(g, gr, prec)


@pytest.mark.parametrize("n,L,seed", [(16, 7, 40), (18, 8, 45), (20, 8, 42)])
@pytest.mark.parametrize("prec", [0, 2])
def test_split_windows_random_local(tlq, n, L, seed, prec):
    # windows of 13 to 16 qubits whose end qubit carries only first-layer gates run as two
    # branches (in shared memory, or on the global tier from 15 up); the first layer draws RX
    # or RY per qubit and RZ / RZZ / CZ at random, so the branch's top rotation gradient (both
    # kinds) and its diagonal terms are exercised, and windows are mirrored where only the
    # bottom end is free
    from paper_2112_10239_gb300 import binding as B
    prob = W.random_local_problem(n, L, 2, seed)
    c, h = tlq.problem(prob)
    try:
        split = B.tlq_plan_cone_stats(tlq.h, c.h, h.h, len(prob.terms))[6]
    finally:
        c.close()
        h.close()
    assert split.sum() > 0
    E, g = _run(tlq, prob, prec=prec)
    Er, gr = _oracle(prob, prob.theta)
    check_energy(E, Er, prec)
    check_grad(g, gr, prec)
    Ee, _ = _run(tlq, prob, prec=prec, grad=False)
    check_energy(Ee, Er, prec)


def test_split_windows_tfim_counts(tlq):
    # n=20, L=6: all eight 13-qubit windows split (the last one laid out mirrored: its top end
    # is the end of the chain, which carries terms); the oracle checks energy and gradient
    from paper_2112_10239_gb300 import binding as B
    prob = W.tfim_n20_L6_B64(B=2)
    c, h = tlq.problem(prob)
    try:
        _, _, _, weff, _, _, split = B.tlq_plan_cone_stats(tlq.h, c.h, h.h, len(prob.terms))
    finally:
        c.close()
        h.close()
    assert list(weff) == [13] * 8 and split.sum() == 8
    E, g = _run(tlq, prob)
    Er, gr = _oracle(prob, prob.theta)
    check_energy(E, Er)
    check_grad(g, gr)


@pytest.mark.parametrize("n,L,B", [(1, 1, 2), (2, 3, 1), (5, 2, 5), (9, 4, 3), (12, 5, 2)])
def test_tfim_small_and_degenerate(tlq, n, L, B):
    prob = W.tfim_problem(n, L, B, seed=n * 10 + L, h_range=(0.5, 1.5))
    E, g = _run(tlq, prob)
    Er, gr = _oracle(prob, prob.theta)
    check_energy(E, Er)
    check_grad(g, gr)


def test_tfim_n8_L2_energy(tlq):
    prob = W.tfim_n8_L2()
    E, _ = _run(tlq, prob, grad=False)
    Er, _ = _oracle(prob, prob.theta, grad=False)
    check_energy(E, Er)


def test_fixed_angles_and_multisite_terms(tlq):
    # Bell / GHZ constructions with fixed angles through the cone path.
    half = math.pi / 2
    n = 6
    gates = [(W.RY, 0, -1, -1, half)]
    for t in range(1, n):
        gates += [(W.RY, t, -1, -1, half), (W.CZ, t - 1, t, -1, 0.0), (W.RY, t, -1, -1, -half)]
    terms = [(1.0, (0, n - 1), "ZZ"), (0.5, tuple(range(n)), "X" * n), (0.25, (1, 2), "YY"), (0.3, (2,), "X")]
    prob = W.Problem(n=n, gates=gates, n_params=0, terms=terms, theta=np.zeros((1, 0)))
    E, _ = _run(tlq, prob, grad=False)
    Er = dense.energy(n, gates, terms, [0.0])
    check_energy(E, [Er])
    # <ZZ> = 1, <X^n> = (-1)^(n-1), <Y1 Y2> = 0 (GHZ), <X2> = 0
    assert abs(E[0] - (1.0 + 0.5 * (-1) ** (n - 1))) < 1e-5


def test_tfim_n20_L6_B64_full(tlq):
    # the full 64-set batch on the GPU; the oracle checks 8 sampled sets exactly
    prob = W.tfim_n20_L6_B64()
    E, g = _run(tlq, prob)
    assert E.shape == (64,) and g.shape == (64, 240)
    idx = [0, 9, 17, 31, 40, 52, 58, 63]
    Er, gr = _oracle(prob, prob.theta[idx])
    check_energy(E[idx], Er)
    check_grad(g[idx], gr)


def test_tfim_n20_L6_gradient_vs_parameter_shift_and_fd(tlq):
    prob = W.tfim_n20_L6_B64(B=1)
    _, g = _run(tlq, prob)
    params = [0, 7, 19, 20, 33, 100, 139, 200, 219, 239]
    ps = dense.grad_param_shift(prob.n, prob.gates, prob.terms, prob.theta[0], params)
    fd = dense.grad_fd(prob.n, prob.gates, prob.terms, prob.theta[0], params, h=1e-3)
    scale = max(1.0, float(np.max(np.abs(g[0]))))
    assert np.max(np.abs(g[0, params] - ps)) <= 1e-4 * scale
    assert np.max(np.abs(g[0, params] - fd)) <= 1e-4 * scale


def test_tfim_n500_L4_B256_sampled(tlq):
    prob = W.tfim_n500_L4_B256()
    E, g = _run(tlq, prob)
    assert E.shape == (256,) and g.shape == (256, 4000)
    cc = windows.ConeCache(prob.gates, prob.terms)
    for b in (0, 255):
        check_energy(E[b:b + 1], [cc.energy(prob.theta[b])])
    Er, gr = cc.grad(prob.theta[77], prob.n_params)
    check_energy(E[77:78], [Er])
    check_grad(g[77], gr)


def test_wide_cones_global_tier(tlq):
    # L=7: X cones have W=15 and ZZ cones W=14, beyond the shared-memory tier.
    prob = W.tfim_problem(18, 7, 2, seed=5, h_range=(0.5, 1.5))
    E, g = _run(tlq, prob)
    Er, gr = _oracle(prob, prob.theta)
    check_energy(E, Er)
    check_grad(g, gr)


def test_batch_invariance(tlq):
    # a set's result is bit-identical alone and inside a larger batch
    prob = W.tfim_n20_L6_B64(B=16)
    E, g = _run(tlq, prob)
    one = W.Problem(prob.n, prob.gates, prob.n_params, prob.terms, prob.theta[5:6])
    E1, g1 = _run(tlq, one)
    assert E1[0] == E[5]
    assert np.array_equal(g1[0], g[5])


def test_repeated_calls_identical(tlq):
    prob = W.tfim_problem(14, 4, 8, seed=3, h_range=(0.5, 1.5))
    a = _run(tlq, prob)
    b = _run(tlq, prob)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_width14_forward_in_shared_memory(tlq):
    # L=7 with ZZ terms only, energies only: every window is 14 wide and runs in shared
    # memory (whole, or as two 13-qubit branches where the top qubit allows it).
    from paper_2112_10239_gb300 import binding as B
    p = W.tfim_problem(22, 7, 3, seed=8, h_range=(0.5, 1.5))
    prob = W.Problem(p.n, p.gates, p.n_params, [t for t in p.terms if t[2] == "ZZ"], p.theta)
    c, h = tlq.problem(prob)
    _, _, _, weff, _, _, _ = B.tlq_plan_cone_stats(tlq.h, c.h, h.h, len(prob.terms))
    c.close()
    h.close()
    assert max(weff) == 14
    E, _ = _run(tlq, prob, grad=False)
    Er, _ = _oracle(prob, prob.theta, grad=False)
    check_energy(E, Er)


def test_global_tier_many_windows_batch_invariant(tlq):
    # n=60, L=7: about 30 windows of 15 qubits per set on the global-memory tier. A 12-set batch
    # has more of them than CTAs (two per SM), so CTAs take several windows in turn; each set
    # must still equal its own single-set call bit for bit. (Correctness of the tier itself
    # against the oracle: test_wide_cones_global_tier.)
    prob = W.tfim_problem(60, 7, 12, seed=21, h_range=(0.5, 1.5))
    E, g = _run(tlq, prob)
    for b in (0, 5, 11):
        one = W.Problem(prob.n, prob.gates, prob.n_params, prob.terms, prob.theta[b:b + 1])
        E1, g1 = _run(tlq, one)
        assert E1[0] == E[b]
        assert np.array_equal(g1[0], g[b])
    assert np.all(np.isfinite(E)) and np.all(np.isfinite(g))


def test_widest_cones_L9(tlq):
    # L=9: X windows of 2L+1 = 19 qubits (the cone path takes up to 20), on the global tier,
    # against the full-chain oracle at n=22 (energy and gradient)
    from paper_2112_10239_gb300 import binding as B
    prob = W.tfim_problem(22, 9, 1, seed=17, h_range=(0.5, 1.5))
    c, h = tlq.problem(prob)
    try:
        _, _, _, weff, _, _, _ = B.tlq_plan_cone_stats(tlq.h, c.h, h.h, len(prob.terms))
    finally:
        c.close()
        h.close()
    assert max(weff) == 19
    E, g = _run(tlq, prob)
    Er, gr = _oracle(prob, prob.theta)
    check_energy(E, Er)
    check_grad(g, gr)


@pytest.mark.parametrize("n,L,width", [(15, 8, 15), (17, 8, 17), (19, 9, 19), (20, 10, 20)])
def test_tiled_global_tier_every_width(tlq, n, L, width):
    # Whole-chain windows give global-tier states of 15, 17, 19 and 20 qubits; with the 14-, 16-
    # and 18-qubit states of the tests above, every sweep plan of the tiled global tier (one or
    # two high register groups, a low sweep with a lone bit 12) runs. Energy only and energy +
    # gradient against the oracle, two parameter sets.
    from paper_2112_10239_gb300 import binding as B
    prob = W.tfim_problem(n, L, 2, seed=30 + n, h_range=(0.5, 1.5))
    c, h = tlq.problem(prob)
    try:
        _, _, _, weff, _, _, split = B.tlq_plan_cone_stats(tlq.h, c.h, h.h, len(prob.terms))
    finally:
        c.close()
        h.close()
    assert width in set((weff - split).tolist())
    Er, gr = _oracle(prob, prob.theta)
    E0, _ = _run(tlq, prob, grad=False)
    check_energy(E0, Er)
    E, g = _run(tlq, prob)
    check_energy(E, Er)
    check_grad(g, gr)
