"""GB300-native expectation-value and gradient engine for layered variational circuits
(the contraction hot path of TensorLy-Quantum, arXiv:2112.10239).

The compute runs in the CUDA library ``libtlq.so`` built from ``csrc/``; ``binding``
wraps its C-ABI with ctypes and ``autograd`` exposes it to PyTorch. ``workloads``
holds the seeded synthetic inputs.
"""
__all__ = ["binding", "workloads"]
