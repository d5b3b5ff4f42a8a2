"""Serving loop (tlq_submit / tlq_poll): continuous batching through the C-ABI.

Each result must be the same alone and in a mix of concurrent requests of different n,
depth and mode, equal to the synchronous call, and match the CPU oracle.
"""
import threading

import numpy as np
import pytest

from oracle import dense
from paper_2112_10239_gb300 import workloads as W
from parity import check_energy, check_grad

pytestmark = pytest.mark.gpu


def _requests(count, seed, n_range=(4, 40), L_range=(1, 5), B_max=3):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        L = int(rng.integers(L_range[0], L_range[1] + 1))
        Bs = int(rng.integers(1, B_max + 1))
        p = W.tfim_problem(n, L, Bs, int(rng.integers(1 << 30)), h_range=(0.5, 1.5))
        out.append((p, bool(rng.random() < 0.4)))
    return out


def _submit(B, ctx, handles, prob, want_grad):
    c, h = handles
    E = np.full(prob.B, np.nan)
    G = np.full(prob.theta.shape, np.nan) if want_grad else None
    th = np.ascontiguousarray(prob.theta)
    t = B.tlq_submit(ctx.h, c.h, h.h, th, E, G)
    return t, (th, E, G)


def _wait(B, ctx, t):
    s = B.tlq_poll(ctx.h, t, -1)
    assert s == B.TLQ_OK


def test_single_request_equals_sync_call(tlq):
    from paper_2112_10239_gb300 import binding as B
    prob = W.tfim_problem(24, 4, 3, seed=9, h_range=(0.5, 1.5))
    handles = tlq.problem(prob)
    t, (th, E, G) = _submit(B, tlq, handles, prob, True)
    _wait(B, tlq, t)
    Es, Gs = B.tlq_expectation_grad(tlq.h, handles[0].h, handles[1].h, prob.theta)
    assert np.array_equal(E, Es) and np.array_equal(G, Gs)
    for hd in handles:
        hd.close()


def test_split_windows_served_equal_sync(tlq):
    # depth 6 and 7: 13- and 15-qubit windows run as two branches each; served alone and
    # together (energy-only and gradient requests), the results equal the synchronous calls
    from paper_2112_10239_gb300 import binding as B
    probs = [W.tfim_problem(24, 6, 2, seed=31, h_range=(0.5, 1.5)),
             W.tfim_problem(20, 7, 1, seed=32, h_range=(0.5, 1.5)),
             W.tfim_problem(17, 6, 3, seed=33, h_range=(0.5, 1.5))]
    grads = [True, True, False]
    handles = [tlq.problem(p) for p in probs]
    for p, hd in zip(probs, handles):
        split = B.tlq_plan_cone_stats(tlq.h, hd[0].h, hd[1].h, len(p.terms))[6]
        assert split.sum() > 0
    pending = [_submit(B, tlq, hd, p, g) for p, g, hd in zip(probs, grads, handles)]
    for t, _ in pending:
        _wait(B, tlq, t)
    for p, g, hd, (_, (th, E, G)) in zip(probs, grads, handles, pending):
        if g:
            Es, Gs = B.tlq_expectation_grad(tlq.h, hd[0].h, hd[1].h, p.theta)
            assert np.array_equal(E, Es) and np.array_equal(G, Gs)
        else:
            Es = B.tlq_expectation(tlq.h, hd[0].h, hd[1].h, p.theta)
            assert np.array_equal(E, Es)
        Er = [dense.energy(p.n, p.gates, p.terms, t) for t in p.theta]
        check_energy(E, Er)
    for hd in handles:
        for x in hd:
            x.close()


def test_alone_and_in_mix_identical(tlq):
    from paper_2112_10239_gb300 import binding as B
    reqs = _requests(40, seed=3)
    handles = [tlq.problem(p) for p, _ in reqs]
    # alone: one request in flight at a time
    alone = []
    for (p, g), hd in zip(reqs, handles):
        t, bufs = _submit(B, tlq, hd, p, g)
        _wait(B, tlq, t)
        alone.append(bufs)
    # mixed: everything submitted at once, batched with each other
    pending = [_submit(B, tlq, hd, p, g) for (p, g), hd in zip(reqs, handles)]
    for t, _ in pending:
        _wait(B, tlq, t)
    for (p, g), a, (_, m) in zip(reqs, alone, pending):
        assert np.array_equal(a[1], m[1])
        if g:
            assert np.array_equal(a[2], m[2])
    # and both agree with the oracle (small ones checked in full)
    for (p, g), a in zip(reqs, alone):
        if p.n > 14:
            continue
        for b in range(p.B):
            if g:
                Er, gr = dense.grad_adjoint(p.n, p.gates, p.terms, p.theta[b], p.n_params)
                check_grad(a[2][b], gr)
            else:
                Er = dense.energy(p.n, p.gates, p.terms, p.theta[b])
            check_energy(a[1][b:b + 1], [Er])
    n, p50, p99, mb = B.tlq_serving_stats(tlq.h)
    assert n >= 80 and 0 < p50 <= p99 and mb >= 1.0
    for hd in handles:
        for x in hd:
            x.close()


def test_wide_cones_in_batch(tlq):
    # L = 7, 8 cones (width 14-17) run on the global-memory tier inside a batch
    from paper_2112_10239_gb300 import binding as B
    probs = [W.tfim_problem(18, 7, 1, seed=1, h_range=(0.5, 1.5)), W.tfim_problem(20, 8, 1, seed=2),
             W.tfim_problem(10, 2, 2, seed=3)]
    handles = [tlq.problem(p) for p in probs]
    pend = [_submit(B, tlq, hd, p, True) for p, hd in zip(probs, handles)]
    for t, _ in pend:
        _wait(B, tlq, t)
    for p, (_, (th, E, G)) in zip(probs, pend):
        for b in range(p.B):
            Er, gr = dense.grad_adjoint(p.n, p.gates, p.terms, p.theta[b], p.n_params)
            check_energy(E[b:b + 1], [Er])
            check_grad(G[b], gr)
    for hd in handles:
        for x in hd:
            x.close()


def test_concurrent_submitters(tlq):
    from paper_2112_10239_gb300 import binding as B
    reqs = _requests(24, seed=5, n_range=(16, 120), L_range=(2, 6), B_max=1)
    handles = [tlq.problem(p) for p, _ in reqs]
    ref = [B.tlq_expectation(tlq.h, hd[0].h, hd[1].h, p.theta) for (p, _), hd in zip(reqs, handles)]
    results = [None] * len(reqs)

    def worker(k):
        for i in range(k, len(reqs), 4):
            p, _ = reqs[i]
            t, bufs = _submit(B, tlq, handles[i], p, False)
            _wait(B, tlq, t)
            results[i] = bufs[1]

    ths = [threading.Thread(target=worker, args=(k,)) for k in range(4)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    for r, e in zip(results, ref):
        assert np.array_equal(r, e)
    for hd in handles:
        for x in hd:
            x.close()


def test_poll_semantics(tlq):
    from paper_2112_10239_gb300 import binding as B
    with pytest.raises(B.TLQError) as ei:
        B.tlq_poll(tlq.h, 987654321, 0)
    assert ei.value.status == B.TLQ_EINVAL
    prob = W.tfim_problem(200, 6, 8, seed=1)
    hd = tlq.problem(prob)
    t, bufs = _submit(B, tlq, hd, prob, True)
    s = B.tlq_poll(tlq.h, t, 0)
    assert s in (B.TLQ_OK, B.TLQ_EAGAIN)
    if s != B.TLQ_OK:
        _wait(B, tlq, t)
    with pytest.raises(B.TLQError):
        B.tlq_poll(tlq.h, t, 0)   # retired
    assert np.all(np.isfinite(bufs[1])) and np.all(np.isfinite(bufs[2]))
    for x in hd:
        x.close()


def test_admission_budget_and_unsupported():
    from paper_2112_10239_gb300 import binding as B
    small = B.Context(device=0, mem_budget=1 << 20)   # 1 MiB: forced-small admission budget
    try:
        prob = W.tfim_n20_L6_B64()
        hd = small.problem(prob)
        E = np.zeros(prob.B)
        G = np.zeros(prob.theta.shape)
        th = np.ascontiguousarray(prob.theta)
        t = B.tlq_submit(small.h, hd[0].h, hd[1].h, th, E, G)
        with pytest.raises(B.TLQError) as ei:
            B.tlq_poll(small.h, t, -1)
        assert ei.value.status == B.TLQ_ENOMEM
        q = W.qaoa_problem(10, 1, 1, seed=0)   # non-local: dense path, not served
        hq = small.problem(q)
        thq = np.ascontiguousarray(q.theta)
        Eq = np.zeros(1)
        t = B.tlq_submit(small.h, hq[0].h, hq[1].h, thq, Eq, None)
        with pytest.raises(B.TLQError) as ei:
            B.tlq_poll(small.h, t, -1)
        assert ei.value.status == B.TLQ_EUNSUPPORTED
        with pytest.raises(B.TLQError) as ei:
            B.tlq_poll(small.h, t, 0)   # failed tickets are retired too
        assert ei.value.status == B.TLQ_EINVAL
    finally:
        small.close()
