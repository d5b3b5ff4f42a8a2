"""CPU ORACLE -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package. It shares no code with the CUDA path and imports nothing from it.

Layout:
  * ``sv_oracle.c``  -- complex128 dense statevector, gate by gate, with its own adjoint
                        gradient (the definition of <H> and nabla <H>, TensorLy-Quantum Sec. 3).
  * ``dense``        -- ctypes binding plus the parameter-shift and finite-difference
                        gradients built on the plain energy.
  * ``windows``      -- per-term light-cone windows for nearest-neighbour circuits that are
                        too wide for a full statevector (naive gate-by-gate support tracking).
  * ``ed``           -- exact diagonalisation with an explicit 2^n x 2^n Hamiltonian (n <= 10).
  * ``density``      -- reduced density operators of pure states (the partial trace by its
                        definition, TensorLy-Quantum Sec. 2 / Sec. 3).
"""
from .dense import (energy, energy_terms, grad_adjoint, grad_param_shift, grad_fd,
                    statevector, pauli_expectation)
from . import windows, ed, density

__all__ = ["energy", "energy_terms", "grad_adjoint", "grad_param_shift", "grad_fd",
           "statevector", "pauli_expectation", "windows", "ed", "density"]
