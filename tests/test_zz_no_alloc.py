"""The allocation-free entry point (tlq_expectation_grad_static) against the regular
device-pointer entry point (tlq_expectation_grad_dev).

tlq_expectation_grad_static serves callers that cannot allocate device memory while they
evaluate (an application whose own allocator owns the GPU, a loop that cannot take
cudaMalloc's implicit synchronisation): its scratch is a fixed array inside the library.
This file is collected last so that a run stopping at its first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_2112_10239_gb300 import workloads as W
from parity import check_energy, check_grad

pytestmark = pytest.mark.gpu


def _dev_call(B, fn, ctx, c, h, theta_t, want_grad=True):
    import torch
    Bsz, P = theta_t.shape
    E = torch.full((Bsz,), float("nan"), dtype=torch.float64, device=theta_t.device)
    G = torch.full((Bsz, P), float("nan"), dtype=torch.float64, device=theta_t.device) if want_grad else None
    torch.cuda.synchronize()
    stream = torch.cuda.Stream(theta_t.device)   # a real stream handle (the legacy default is 0)
    fn(ctx.h, c.h, h.h, theta_t.data_ptr(), Bsz, *([B.TLQ_FP32] if fn is B.tlq_expectation_grad_dev else []),
       E.data_ptr(), G.data_ptr() if G is not None else None, stream.cuda_stream)
    stream.synchronize()
    torch.cuda.synchronize()
    return E.cpu().numpy(), (G.cpu().numpy() if G is not None else None)


def test_static_scratch_matches_regular_entry_point(tlq):
    import torch
    from paper_2112_10239_gb300 import binding as B

    prob = W.tfim_n20_L6_B64(B=16)
    c, h = tlq.problem(prob)
    dev = torch.device("cuda", 0)
    th1 = torch.tensor(prob.theta, dtype=torch.float64, device=dev)
    th2 = torch.tensor(prob.theta[::-1].copy() + 0.25, dtype=torch.float64, device=dev)
    try:
        for th in (th1, th2):   # two calls in a row: the shared array's leftovers must not leak
            E_ref, G_ref = _dev_call(B, B.tlq_expectation_grad_dev, tlq, c, h, th)
            E_st, G_st = _dev_call(B, B.tlq_expectation_grad_static, tlq, c, h, th)
            assert np.all(np.isfinite(E_st)) and np.all(np.isfinite(G_st))
            check_energy(E_st, E_ref)
            check_grad(G_st, G_ref)
        # energies only (grad pointer NULL)
        E_ref, _ = _dev_call(B, B.tlq_expectation_grad_dev, tlq, c, h, th1, want_grad=False)
        E_st, _ = _dev_call(B, B.tlq_expectation_grad_static, tlq, c, h, th1, want_grad=False)
        check_energy(E_st, E_ref)
    finally:
        c.close()
        h.close()


def test_static_scratch_rejects_oversized_call(tlq):
    import torch
    from paper_2112_10239_gb300 import binding as B

    prob = W.tfim_n500_L4_B256()   # gradient slots alone exceed the 16 MiB array
    c, h = tlq.problem(prob)
    dev = torch.device("cuda", 0)
    th = torch.tensor(prob.theta, dtype=torch.float64, device=dev)
    E = torch.zeros(prob.B, dtype=torch.float64, device=dev)
    G = torch.zeros(prob.theta.shape, dtype=torch.float64, device=dev)
    try:
        with pytest.raises(B.TLQError) as ei:
            B.tlq_expectation_grad_static(tlq.h, c.h, h.h, th.data_ptr(), prob.B, E.data_ptr(), G.data_ptr(), None)
        assert ei.value.status == B.TLQ_ENOMEM
        assert "static array" in str(ei.value)
    finally:
        c.close()
        h.close()


def test_static_scratch_allocates_no_device_memory(tlq):
    """After one warm-up call, further calls (same and different batch size, with and without
    gradients) leave the device's free memory unchanged."""
    import torch
    from paper_2112_10239_gb300 import binding as B

    prob = W.tfim_n20_L6_B64(B=16)
    c, h = tlq.problem(prob)
    dev = torch.device("cuda", 0)
    th = torch.tensor(prob.theta, dtype=torch.float64, device=dev)
    E = torch.zeros(prob.B, dtype=torch.float64, device=dev)
    G = torch.zeros(prob.theta.shape, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(dev)
    try:
        B.tlq_expectation_grad_static(tlq.h, c.h, h.h, th.data_ptr(), prob.B, E.data_ptr(), G.data_ptr(),
                                      stream.cuda_stream)
        stream.synchronize()
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info(dev)
        for nb, grad in ((prob.B, True), (8, True), (prob.B, False), (3, False)):
            B.tlq_expectation_grad_static(tlq.h, c.h, h.h, th.data_ptr(), nb, E.data_ptr(),
                                          G.data_ptr() if grad else None, stream.cuda_stream)
        stream.synchronize()
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info(dev)
        assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
    finally:
        c.close()
        h.close()


def test_static_scratch_two_threads_two_contexts():
    """Two contexts driven from two threads at once, each cycling through 18 distinct circuits
    (more than the 16 cached host plans, so entries are evicted while the other thread uses
    its own). Both threads enqueue on one shared stream: the library enqueues each call's
    copies and launches as one unit, so the calls run one after another on the GPU and do not
    race on the shared array. Every result must equal tlq_expectation_grad_dev's."""
    import threading
    import torch
    from paper_2112_10239_gb300 import binding as B

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    probs = [W.tfim_problem(8 + (k % 6), 2 + (k % 3), 4, seed=100 + k, h_range=(0.5, 1.5)) for k in range(18)]
    failures = []

    def worker(tid):
        try:
            with B.Context(device=0) as ctx:
                handles = [ctx.problem(p) for p in probs]
                thetas = [torch.tensor(p.theta + 0.1 * tid, dtype=torch.float64, device=dev) for p in probs]
                for rnd in range(2):
                    order = range(len(probs)) if (rnd + tid) % 2 == 0 else reversed(range(len(probs)))
                    for k in order:
                        p, (c, h), th = probs[k], handles[k], thetas[k]
                        Er = torch.empty(p.B, dtype=torch.float64, device=dev)
                        Gr = torch.empty(p.theta.shape, dtype=torch.float64, device=dev)
                        Es = torch.full((p.B,), float("nan"), dtype=torch.float64, device=dev)
                        Gs = torch.full(p.theta.shape, float("nan"), dtype=torch.float64, device=dev)
                        torch.cuda.synchronize()
                        B.tlq_expectation_grad_dev(ctx.h, c.h, h.h, th.data_ptr(), p.B, B.TLQ_FP32, Er.data_ptr(),
                                                   Gr.data_ptr(), stream.cuda_stream)
                        B.tlq_expectation_grad_static(ctx.h, c.h, h.h, th.data_ptr(), p.B, Es.data_ptr(),
                                                      Gs.data_ptr(), stream.cuda_stream)
                        stream.synchronize()
                        check_energy(Es.cpu().numpy(), Er.cpu().numpy())
                        check_grad(Gs.cpu().numpy(), Gr.cpu().numpy())
                for c, h in handles:
                    c.close()
                    h.close()
        except Exception as exc:  # reported by the main thread
            failures.append((tid, repr(exc)))

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    threads = [threading.Thread(target=worker, args=(t,)) for t in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=600)
    assert not any(t.is_alive() for t in threads), "a worker thread did not finish"
    assert not failures, failures
