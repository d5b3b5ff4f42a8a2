"""Host-side checks of the C-ABI library (no GPU): it loads, exports every symbol that
include/tlq.h declares, validates descriptors, and plans the exact causal cones."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2112_10239_gb300 import build as tlq_build
from paper_2112_10239_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    tlq_build.build()
    from paper_2112_10239_gb300 import binding
    return binding


@pytest.fixture()
def hctx(B):
    ctx = B.Context(device=-1)
    yield ctx
    ctx.close()


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "tlq.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(tlq_[a-z_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(B):
    L = B.lib()
    syms = header_symbols()
    assert len(syms) >= 14
    for s in syms:
        assert hasattr(L, s), s
    assert sorted(B.SYMBOLS) == syms
    assert B.tlq_version() == 10000


def test_struct_layout_matches_header(B):
    # tlq_gate: 4 x int32 + double = 24 bytes; tlq_term: double, int32, 2 pointers.
    assert ctypes.sizeof(B.tlq_gate) == 24
    assert B.tlq_term.sites.offset == 16


def _err(B, fn, *a):
    with pytest.raises(B.TLQError) as ei:
        fn(*a)
    return ei.value.status


def test_circuit_validation(B, hctx):
    ok = [(W.RY, 0, -1, 0, 0.0), (W.CZ, 0, 1, -1, 0.0)]
    c = hctx.circuit(2, ok, 1)
    c.close()
    bad = [
        ([(W.RY, 2, -1, 0, 0.0)], 1),          # qubit out of range
        ([(W.CZ, 0, 0, -1, 0.0)], 1),          # q0 == q1
        ([(W.RZZ, 0, 5, 0, 0.0)], 1),          # second qubit out of range
        ([(W.RY, 0, -1, 1, 0.0)], 1),          # param >= n_params
        ([(W.RY, 0, -1, -2, 0.0)], 1),         # param < -1
        ([(9, 0, -1, 0, 0.0)], 1),             # unknown kind
    ]
    for gates, P in bad:
        assert _err(B, B.tlq_circuit_create, hctx.h, 2, gates, P) == B.TLQ_EINVAL
    assert _err(B, B.tlq_circuit_create, hctx.h, 0, ok, 1) == B.TLQ_EINVAL


def test_hamiltonian_validation(B, hctx):
    h = hctx.hamiltonian(3, [(1.0, (0, 1), "ZZ"), (0.5, (2,), "X")])
    h.close()
    for terms in ([(1.0, (0, 3), "ZZ")], [(1.0, (0,), "Q")], [(1.0, (1, 1), "ZZ")], [(1.0, (), "")]):
        assert _err(B, B.tlq_hamiltonian_create, hctx.h, 3, terms) == B.TLQ_EINVAL
    assert _err(B, B.tlq_hamiltonian_create, hctx.h, 3, []) == B.TLQ_EINVAL


def test_host_only_context_refuses_compute(B, hctx):
    p = W.tfim_n8_L2()
    c, h = hctx.problem(p)
    assert _err(B, B.tlq_expectation, hctx.h, c.h, h.h, p.theta) == B.TLQ_EUNSUPPORTED
    # mismatched qubit counts
    h2 = hctx.hamiltonian(9, [(1.0, (0,), "Z")])
    assert _err(B, B.tlq_expectation, hctx.h, c.h, h2.h, p.theta) == B.TLQ_EINVAL


@pytest.mark.parametrize("n,L", [(8, 2), (20, 6), (40, 4), (30, 7)])
def test_planner_exact_cone_widths(B, hctx, n, L):
    # ZZ terms: 2L sites, X terms: 2L+1 sites, clipped at the chain ends.
    p = W.tfim_problem(n, L, 1, seed=0)
    c, h = hctx.problem(p)
    path, lo, w, ng = B.tlq_plan_info(hctx.h, c.h, h.h, len(p.terms))
    assert path == B.TLQ_PATH_CONE
    for t, (_, sites, letters) in enumerate(p.terms):
        i = sites[0]
        if letters == "ZZ":
            want_lo, want_hi = max(0, i - (L - 1)), min(n - 1, i + 1 + (L - 1))
        else:
            want_lo, want_hi = max(0, i - L), min(n - 1, i + L)
        assert (lo[t], lo[t] + w[t] - 1) == (want_lo, want_hi), (t, letters)


def test_planner_window_inside_oracle_window(B, hctx):
    # The oracle's plain gate-by-gate light cone is a superset of the exact cone.
    from oracle import windows
    p = W.random_local_problem(16, 3, 1, seed=4)
    c, h = hctx.problem(p)
    path, lo, w, ng = B.tlq_plan_info(hctx.h, c.h, h.h, len(p.terms))
    assert path == B.TLQ_PATH_CONE
    for t, (_, sites, _) in enumerate(p.terms):
        qubits, keep = windows.cone(p.gates, sites)
        assert min(qubits) <= lo[t] and lo[t] + w[t] - 1 <= max(qubits)
        assert ng[t] <= len(keep)


@pytest.mark.parametrize("n,L,n_split", [(20, 6, 8), (500, 4, 0), (100, 7, 86), (100, 8, 84)])
def test_planner_window_branches(B, hctx, n, L, n_split):
    # Windows of 13 or more qubits whose end qubit carries only first-layer gates and no term
    # run as two branches; in the brick-wall Ising circuits that is every wide window (the
    # clipped one at the chain's top end laid out mirrored). Each window measures at most 16
    # terms and every term exactly once.
    p = W.tfim_problem(n, L, 1, seed=0)
    c, h = hctx.problem(p)
    nrot, ndiag, npdiag, weff, wtrue, nterms, split = B.tlq_plan_cone_stats(hctx.h, c.h, h.h, len(p.terms))
    assert int(split.sum()) == n_split
    assert np.all(split[weff < 13] == 0) and np.all(split[weff >= 13] == 1)
    assert np.all(wtrue[split == 1] == weff[split == 1])
    assert nterms.max() <= 16 and int(nterms.sum()) == len(p.terms)


def test_planner_no_branches_when_both_ends_are_measured(B, hctx):
    # an X X term on both ends of a 13-qubit chain: the whole-chain window has terms on its
    # top and bottom qubit, so it cannot be split either way
    p = W.tfim_problem(13, 6, 1, seed=0)
    p = W.Problem(p.n, p.gates, p.n_params, p.terms + [(0.7, (0, 12), "XX")], p.theta)
    c, h = hctx.problem(p)
    weff, split = B.tlq_plan_cone_stats(hctx.h, c.h, h.h, len(p.terms))[3::3]
    assert 13 in list(weff) and int(split.sum()) == 0


def test_non_local_circuit_goes_dense(B, hctx):
    p = W.qaoa_problem(10, 2, 1, seed=0)
    c, h = hctx.problem(p)
    path, *_ = B.tlq_plan_info(hctx.h, c.h, h.h, len(p.terms))
    assert path == B.TLQ_PATH_DENSE


def test_dense_plan_info(B, hctx):
    # n=28, p=4 QAOA: 28 qubits, the first layer's RZZ is a phase on |0..0> (dropped); each
    # layer's RX touches all 28 qubits: a low tile (0..11) and two strided tiles (12..19, 20..27)
    p = W.qaoa_n28_p4()
    c, h = hctx.problem(p)
    n_eff, n_passes, n_fwd, n_rev_store, n_x, fused = B.tlq_plan_dense_info(hctx.h, c.h, h.h)
    assert (n_eff, n_x, fused) == (28, 0, 1)
    assert 4 <= n_passes <= 12          # at least one pass per layer, at most three
    assert 3 <= n_fwd < n_passes        # layers 1..3 after the product-state start
    assert n_rev_store <= n_passes - 2  # the first pass and layer-0-only passes write nothing
    # small circuits keep a 12-qubit state (one tile); X/Y strings are measured separately
    q = W.random_nonlocal_problem(6, 2, 1, seed=1)
    c2, h2 = hctx.problem(q)
    n_eff, _, _, _, n_x, _ = B.tlq_plan_dense_info(hctx.h, c2.h, h2.h)
    assert n_eff == 12
    assert n_x == sum(1 for _, _, letters in q.terms if set(letters) - {"Z"})


def test_dense_plan_bytes(B, hctx):
    # the schedule's HBM traffic, recounted from the pass counts: the n=28 QAOA forward starts in
    # a low tile at bit 0, so its first pass generates layer 0's state (no start write, no first
    # read) and an energy without X/Y terms skips the last write; the tensor-core passes keep the
    # start kernel
    p = W.qaoa_n28_p4()
    c, h = hctx.problem(p)
    n_eff, n_passes, n_fwd, n_rev_store, n_x, _ = B.tlq_plan_dense_info(hctx.h, c.h, h.h)
    S = 8.0 * 2 ** n_eff
    assert B.tlq_plan_dense_bytes(hctx.h, c.h, h.h, False) == (2 * n_fwd - 2) * S
    assert B.tlq_plan_dense_bytes(hctx.h, c.h, h.h, False, B.TLQ_MIXED_TC) == (2 * n_fwd) * S
    grad = (2 * n_fwd - 1) * S + S + 2 * n_passes * S + 2 * n_rev_store * S
    assert B.tlq_plan_dense_bytes(hctx.h, c.h, h.h, True) == grad
    # X/Y terms: one read each, and the last forward write stays (the terms read the final state)
    q = W.random_nonlocal_problem(14, 2, 1, seed=3)
    c2, h2 = hctx.problem(q)
    n_eff, n_passes, n_fwd, n_rev_store, n_x, _ = B.tlq_plan_dense_info(hctx.h, c2.h, h2.h)
    assert n_x > 0
    S = 8.0 * 2 ** n_eff
    e = B.tlq_plan_dense_bytes(hctx.h, c2.h, h2.h, False)
    assert e in ((2 * n_fwd - 1 + n_x) * S, (2 * n_fwd + 1 + n_x) * S)   # with or without the start kernel


def test_partial_trace_argument_checks(B, hctx):
    # validation happens before any device work: EINVAL for bad kept-qubit lists, then the
    # host-only context reports EUNSUPPORTED for a valid request
    import ctypes
    L = B.lib()
    ip = ctypes.POINTER(ctypes.c_int32)

    def pt(n, keep):
        k = np.array(keep, dtype=np.int32)
        return L.tlq_partial_trace_dev(hctx.h, ctypes.c_void_p(16), n, k.ctypes.data_as(ip), len(keep),
                                       ctypes.c_void_p(16), None)

    assert pt(10, [0, 10]) == B.TLQ_EINVAL          # out of range
    assert pt(10, [3, 3]) == B.TLQ_EINVAL           # repeated
    assert pt(10, []) == B.TLQ_EINVAL               # m = 0
    assert pt(32, [0]) == B.TLQ_EINVAL              # n > 31
    assert pt(20, list(range(16))) == B.TLQ_EINVAL  # m > 15
    assert pt(10, [7, 2]) == B.TLQ_EUNSUPPORTED     # valid; host-only context
    p = W.tfim_problem(500, 4, 1, seed=6)
    c, h = hctx.problem(p)
    th = np.ascontiguousarray(p.theta[0])
    rho = np.zeros(2 * 64)
    dp = ctypes.POINTER(ctypes.c_double)

    def rd(keep):
        k = np.array(keep, dtype=np.int32)
        return L.tlq_reduced_density(hctx.h, c.h, th.ctypes.data_as(dp), k.ctypes.data_as(ip), len(keep),
                                     rho.ctypes.data_as(dp))

    assert rd([499, 500]) == B.TLQ_EINVAL
    assert rd(list(range(15))) == B.TLQ_EINVAL      # the host API returns at most 14 kept qubits
    assert rd([250, 251, 253]) == B.TLQ_EUNSUPPORTED


@pytest.mark.parametrize("n,L", [(1, 2), (2, 1), (8, 2), (20, 6), (500, 4)])
def test_mps_plan_bond_dimensions(B, hctx, n, L):
    # the brick-wall puts one CZ per layer on every neighbouring pair: 2^L bond dimension on
    # every inner bond; per set the plan holds the site tensors (2 chi_l chi_r each), four
    # environments per bond (chi^2 each) and two chains per bond inside each term's span
    p = W.tfim_problem(n, L, 1, seed=0)
    c, h = hctx.problem(p)
    bits, elems, fe, fg = B.tlq_plan_mps_info(hctx.h, c.h, h.h)
    assert bits == (L if n > 1 else 0)
    assert 0 < fe < fg
    chi = [1] + [2 ** L] * (n - 1) + [1]
    a = sum(2 * chi[q] * chi[q + 1] for q in range(n))
    env = sum(x * x for x in chi)
    chain = sum(chi[k] ** 2 for _, s, _ in p.terms for k in range(min(s) + 1, max(s) + 1))
    assert elems == a + 4 * env + 2 * chain


def test_mps_plan_counts_gates_per_pair(B, hctx):
    # bonds count the two-qubit gates on each pair, in either qubit order, RZZ and CZ alike
    gates = [(W.RY, 0, -1, 0, 0.0), (W.CZ, 1, 0, -1, 0.0), (W.RZZ, 0, 1, 1, 0.0), (W.RZZ, 2, 1, 2, 0.0)]
    c = hctx.circuit(3, gates, 3)
    h = hctx.hamiltonian(3, [(1.0, (0, 2), "XZ")])
    bits, elems, _, _ = B.tlq_plan_mps_info(hctx.h, c.h, h.h)
    chi = [1, 4, 2, 1]
    assert bits == 2
    assert elems == (2 * (1 * 4 + 4 * 2 + 2 * 1) + 4 * (1 + 16 + 4 + 1) + 2 * (16 + 4))


def test_mps_plan_limits(B, hctx):
    # non-neighbouring two-qubit gates, more than 6 gates on one pair, more than 48 gates on one
    # qubit: EUNSUPPORTED (the cone and dense paths still take such circuits)
    q = W.qaoa_problem(10, 2, 1, seed=0)
    c, h = hctx.problem(q)
    assert _err(B, B.tlq_plan_mps_info, hctx.h, c.h, h.h) == B.TLQ_EUNSUPPORTED
    hz = hctx.hamiltonian(2, [(1.0, (0, 1), "ZZ")])
    c7 = hctx.circuit(2, [(W.CZ, 0, 1, -1, 0.0)] * 7, 0)
    assert _err(B, B.tlq_plan_mps_info, hctx.h, c7.h, hz.h) == B.TLQ_EUNSUPPORTED
    c6 = hctx.circuit(2, [(W.CZ, 0, 1, -1, 0.0)] * 6, 0)
    assert B.tlq_plan_mps_info(hctx.h, c6.h, hz.h)[0] == 6
    c49 = hctx.circuit(2, [(W.RX, 0, -1, 0, 0.0)] * 49, 1)
    assert _err(B, B.tlq_plan_mps_info, hctx.h, c49.h, hz.h) == B.TLQ_EUNSUPPORTED
    # compute calls need a device
    p = W.tfim_n8_L2()
    c8, h8 = hctx.problem(p)
    assert _err(B, B.tlq_mps_expectation, hctx.h, c8.h, h8.h, p.theta) == B.TLQ_EUNSUPPORTED


@pytest.mark.parametrize("n,L,extra", [(9, 3, False), (12, 2, True)])
def test_mps_flop_count(B, hctx, n, L, extra):
    # the roofline numerator of the MPS route, recounted here from the circuit and the term
    # spans: per site q (bond dimensions dl, dr) the left sweep forms the norm group, the H group
    # (with gradients: H plus the terms ending at q) and one chain per term continuing right;
    # the right sweep the mirror image (chains only with gradients); the site kernel one group
    # per covering term plus two (with gradients) or the terms ending at q (energy only)
    p = W.tfim_problem(n, L, 1, seed=0)
    terms = list(p.terms) + ([(0.5, (1, n - 2), "XZ")] if extra else [])
    c = hctx.circuit(n, p.gates, p.n_params)
    h = hctx.hamiltonian(n, terms)
    _, _, fe, fg = B.tlq_plan_mps_info(hctx.h, c.h, h.h)
    chi = [1] + [2 ** L] * (n - 1) + [1]
    spans = [(min(s), max(s)) for _, s, _ in terms]

    def count(grad):
        cm = 0
        for q in range(n):
            dl, dr = chi[q], chi[q + 1]
            cov = [(i, j) for i, j in spans if i <= q <= j]
            end_l = sum(j == q for i, j in cov)
            end_r = sum(i == q for i, j in cov)
            cont_l, cont_r = len(cov) - end_l, len(cov) - end_r
            ncl, ngl = 1 + (1 + end_l if grad else 0) + cont_l, 1 + (1 if grad else 0) + cont_l
            ncr, ngr = 1 + (1 + end_r + cont_r if grad else 0), 1 + (1 + cont_r if grad else 0)
            cm += ncl * 2 * dl * dr * dl + ngl * 2 * dr * dr * dl
            cm += ncr * 2 * dr * dl * dr + ngr * 2 * dl * dl * dr
            cm += (2 + len(cov) if grad else end_l) * 2 * dl * dr * (dl + dr)
        return 8.0 * cm

    assert fe == count(False) and fg == count(True)
