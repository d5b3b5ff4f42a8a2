"""Per-term light-cone windows for circuits too wide for one statevector.

Test infrastructure only (see the package docstring).

For a Pauli term P on sites S, <0|U^dag P U|0> only involves the gates in P's
backward light cone: walking the gate list from the end, a gate belongs to the cone
when it touches the support collected so far, and then its qubits join the support.
Gates that never touch the support commute past P and cancel against their
adjoints. This is the plain gate-by-gate rule -- it ignores that diagonal gates
commute with each other, so it keeps more qubits than the tightest cone, which is
fine: any superset of the cone gives the exact value. The cone gates are then
simulated on a dense statevector over the support's qubits (relabelled 0..w-1)
with the dense oracle.

The tighter cone used by the CUDA path ("causality-simplified contraction", which
the paper's Sec. 4 names as future work) is not reproduced here, so the two sides
stay independent.
"""
from __future__ import annotations

import numpy as np

from . import dense


def cone(gates, sites):
    """Return (qubits, gate_indices): the sorted support and the cone gates in order."""
    support = set(int(s) for s in sites)
    keep = []
    for k in range(len(gates) - 1, -1, -1):
        kind, q0, q1, _, _ = gates[k]
        qs = (q0,) if q1 < 0 else (q0, q1)
        if any(q in support for q in qs):
            keep.append(k)
            support.update(qs)
    keep.reverse()
    return sorted(support), keep


class ConeCache:
    """Cone structure per term, computed once per (gate list, term list)."""

    def __init__(self, gates, terms):
        self.gates = gates
        self.terms = terms
        self.cones = []
        for (c, sites, letters) in terms:
            qubits, keep = cone(gates, sites)
            relabel = {q: i for i, q in enumerate(qubits)}
            sub = []
            for k in keep:
                kind, q0, q1, p, a = gates[k]
                sub.append((kind, relabel[q0], relabel[q1] if q1 >= 0 else -1, p, a))
            term = (1.0, tuple(relabel[s] for s in sites), letters)
            self.cones.append((len(qubits), sub, term, c))

    def max_width(self):
        return max(w for w, _, _, _ in self.cones)

    def energy_terms(self, theta):
        et = np.zeros(len(self.cones))
        for t, (w, sub, term, _) in enumerate(self.cones):
            et[t] = dense.energy(w, sub, [term], theta)
        E = float(sum(c * e for (_, _, _, c), e in zip(self.cones, et)))
        return E, et

    def energy(self, theta):
        return self.energy_terms(theta)[0]

    def grad(self, theta, n_params):
        E = 0.0
        g = np.zeros(n_params)
        for (w, sub, term, c) in self.cones:
            e_t, g_t = dense.grad_adjoint(w, sub, [term], theta, n_params)
            E += c * e_t
            g += c * g_t
        return E, g
