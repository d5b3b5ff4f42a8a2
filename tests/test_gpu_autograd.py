"""torch.autograd wrapper around the CUDA engine."""
import numpy as np
import pytest

from oracle import dense
from paper_2112_10239_gb300 import workloads as W
from parity import check_energy, check_grad

pytestmark = pytest.mark.gpu


def test_autograd_matches_oracle_and_chain_rule():
    import torch
    from paper_2112_10239_gb300 import binding as B
    from paper_2112_10239_gb300.autograd import Engine, Expectation

    prob = W.tfim_problem(10, 3, 4, seed=2, h_range=(0.5, 1.5))
    eng = Engine(prob.n, prob.gates, prob.n_params, prob.terms)
    try:
        model = Expectation(eng)
        theta = torch.tensor(prob.theta, dtype=torch.float64, device="cuda", requires_grad=True)
        w = torch.tensor([0.5, -1.0, 2.0, 0.25], dtype=torch.float64, device="cuda")
        E = model(theta)
        (w * E).sum().backward()
        Er, gr = zip(*[dense.grad_adjoint(prob.n, prob.gates, prob.terms, th, prob.n_params) for th in prob.theta])
        check_energy(E.detach().cpu().numpy(), np.array(Er))
        want = w.cpu().numpy()[:, None] * np.array(gr)
        check_grad(theta.grad.cpu().numpy(), want)
    finally:
        eng.close()


def test_gradcheck_fp64_reference_mode():
    import torch
    from paper_2112_10239_gb300 import binding as B
    from paper_2112_10239_gb300.autograd import Engine, TLQExpectation

    prob = W.random_local_problem(6, 2, 2, seed=3)
    eng = Engine(prob.n, prob.gates, prob.n_params, prob.terms, prec=B.TLQ_FP64_REF)
    try:
        theta = torch.tensor(prob.theta, dtype=torch.float64, device="cuda", requires_grad=True)
        assert torch.autograd.gradcheck(lambda t: TLQExpectation.apply(t, eng), (theta,), eps=1e-6, atol=1e-6)
    finally:
        eng.close()
