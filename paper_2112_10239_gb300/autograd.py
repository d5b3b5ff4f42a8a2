"""PyTorch autograd wrapper: energies as a differentiable function of the angles.

The forward pass calls ``tlq_expectation_grad_dev`` (TensorLy-Quantum Sec. 3: the expectation
value <H> and, in the same launch, its full gradient from the adjoint sweep) on the current
CUDA stream with device pointers; the backward pass returns ``grad_E[:, None] * dE/dtheta``.
PyTorch only provides the tensors and the stream; all arithmetic runs in ``libtlq.so``.
"""
from __future__ import annotations

import torch

from . import binding as B

_LEGACY_STREAM = 1   # cudaStreamLegacy: torch's default stream has handle 0


class Engine:
    """A context plus one circuit and one Hamiltonian, created once and kept resident."""

    def __init__(self, n, gates, n_params, terms, device=0, prec=B.TLQ_FP32):
        self.ctx = B.Context(device=device)
        self.circ = self.ctx.circuit(n, gates, n_params)
        self.ham = self.ctx.hamiltonian(n, terms)
        self.n_params = n_params
        self.device = torch.device("cuda", device)
        self.prec = prec

    def close(self):
        self.circ.close()
        self.ham.close()
        self.ctx.close()


class TLQExpectation(torch.autograd.Function):
    """E[b] = <psi(theta_b)|H|psi(theta_b)> for theta of shape [B, n_params] (float64, CUDA)."""

    @staticmethod
    def forward(ctx, theta, engine):
        if theta.dim() != 2 or theta.shape[1] != engine.n_params:
            raise ValueError(f"theta must be [B, {engine.n_params}]")
        th = theta.detach().to(device=engine.device, dtype=torch.float64).contiguous()
        Bsz = th.shape[0]
        E = torch.empty(Bsz, dtype=torch.float64, device=engine.device)
        G = torch.empty(Bsz, engine.n_params, dtype=torch.float64, device=engine.device)
        handle = torch.cuda.current_stream(engine.device).cuda_stream or _LEGACY_STREAM
        B.tlq_expectation_grad_dev(engine.ctx.h, engine.circ.h, engine.ham.h, th.data_ptr(), Bsz, engine.prec,
                                   E.data_ptr(), G.data_ptr(), handle)
        ctx.save_for_backward(G)
        return E

    @staticmethod
    def backward(ctx, grad_E):
        (G,) = ctx.saved_tensors
        return grad_E.to(G.dtype)[:, None] * G, None


class Expectation(torch.nn.Module):
    """``Expectation(engine)(theta) -> energies`` with gradients for autograd."""

    def __init__(self, engine: Engine):
        super().__init__()
        self.engine = engine

    def forward(self, theta):
        return TLQExpectation.apply(theta, self.engine)
