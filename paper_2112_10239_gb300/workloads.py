"""Seeded synthetic inputs shared by the tests, the benchmark and the CPU oracle checks.

This module only *describes* inputs: gate lists, Pauli-term lists, angle arrays and
request streams drawn from ``numpy.random.default_rng(seed)`` (PCG64). It holds none
of the simulation arithmetic (no gate matrices, no contraction, no expectation
values), so both the CUDA path and the oracle can consume its output without sharing
method code.

Conventions (readings of the paper, which states none of them):
  * gates are ``(kind, q0, q1, param, angle)`` tuples; ``kind`` is one of
    ``RX, RY, RZ, RZZ, CZ``; ``q1 = -1`` for one-qubit gates; ``param = -1``
    means the fixed ``angle`` is used, otherwise ``theta[param]``;
  * rotations are ``exp(-i angle P / 2)`` and the initial state is ``|0...0>``;
  * qubit ``q`` is bit ``q`` of the amplitude index;
  * Hamiltonians are sums of Pauli strings ``(coeff, sites, letters)`` -- the
    paper's transverse-field Ising model (Sec. 3, the n=500 experiment) is
    ``J sum_i Z_i Z_{i+1} + sum_i h_i X_i`` taken with the literal ``+`` signs;
  * the layered ansatz of the Ising workloads applies, per layer ``l``,
    ``RY(a_{l,q})`` on every qubit, ``RZ(b_{l,q})`` on every qubit, ``CZ`` on the
    even pairs (0,1),(2,3),... then on the odd pairs (1,2),(3,4),... of an open
    chain, with parameter index ``p = l*2n + kind*n + q`` (kind 0 = a, 1 = b).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

RX, RY, RZ, RZZ, CZ = 0, 1, 2, 3, 4
KIND_NAMES = {RX: "RX", RY: "RY", RZ: "RZ", RZZ: "RZZ", CZ: "CZ"}


@dataclass
class Problem:
    """One circuit + Hamiltonian + a batch of angle sets."""

    n: int
    gates: list            # [(kind, q0, q1, param, angle)]
    n_params: int
    terms: list            # [(coeff, (sites...), "letters")]
    theta: np.ndarray      # float64 [B, n_params]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def B(self) -> int:
        return int(self.theta.shape[0])


_BRICKWALL_CACHE: dict = {}


def brickwall_gates(n: int, L: int) -> list:
    """RY/RZ + CZ brick-wall gate list with ``p = l*2n + kind*n + q`` (memoised; treat the
    returned list as read-only)."""
    key = (n, L)
    if key in _BRICKWALL_CACHE:
        return _BRICKWALL_CACHE[key]
    gates = []
    for l in range(L):
        for q in range(n):
            gates.append((RY, q, -1, l * 2 * n + q, 0.0))
        for q in range(n):
            gates.append((RZ, q, -1, l * 2 * n + n + q, 0.0))
        for q in range(0, n - 1, 2):
            gates.append((CZ, q, q + 1, -1, 0.0))
        for q in range(1, n - 1, 2):
            gates.append((CZ, q, q + 1, -1, 0.0))
    _BRICKWALL_CACHE[key] = gates
    return gates


def tfim_terms(n: int, J: float, h) -> list:
    """``J sum_i Z_i Z_{i+1}`` (open chain) followed by ``sum_i h_i X_i``."""
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), (n,))
    terms = [(float(J), (i, i + 1), "ZZ") for i in range(n - 1)]
    terms += [(float(h[i]), (i,), "X") for i in range(n)]
    return terms


def tfim_problem(n: int, L: int, B: int, seed: int, J: float = 1.0,
                 h_range=None, name: str = "") -> Problem:
    """Layered RY/RZ+CZ ansatz against the transverse-field Ising chain.

    RNG order: ``h[n]`` first (only when ``h_range`` is given, uniform in that
    range; otherwise ``h_i = 1``), then ``theta[B][L][2][n]`` uniform in [0, 2pi).
    """
    rng = np.random.default_rng(seed)
    if h_range is not None:
        h = rng.uniform(h_range[0], h_range[1], size=n)
    else:
        h = np.ones(n)
    theta = rng.uniform(0.0, 2.0 * math.pi, size=(B, L, 2, n)).reshape(B, L * 2 * n)
    return Problem(n=n, gates=brickwall_gates(n, L), n_params=2 * n * L,
                   terms=tfim_terms(n, J, h), theta=np.ascontiguousarray(theta),
                   name=name or f"tfim_n{n}_L{L}_B{B}",
                   meta={"L": L, "J": J, "h": h, "layout": "brickwall"})


def random_regular3_graph(n: int, rng: np.random.Generator) -> list:
    """Pairing-model 3-regular graph; self-loops and multi-edges are rejected."""
    if (3 * n) % 2:
        raise ValueError("3-regular graph needs an even vertex count")
    while True:
        stubs = np.repeat(np.arange(n), 3)
        rng.shuffle(stubs)
        pairs = stubs.reshape(-1, 2)
        edges = set()
        ok = True
        for u, v in pairs:
            u, v = int(u), int(v)
            if u == v:
                ok = False
                break
            e = (min(u, v), max(u, v))
            if e in edges:
                ok = False
                break
            edges.add(e)
        if ok:
            return sorted(edges)


def qaoa_problem(n: int, p: int, B: int, seed: int, name: str = "",
                 edges=None) -> Problem:
    """QAOA-style circuit: per layer RZZ(gamma_l) on every edge then RX(beta_l) on
    every qubit; ``H = sum_e Z_u Z_v``; gamma, beta uniform in [0, pi).

    Parameter index: gamma_l = 2l, beta_l = 2l+1 (shared by all edges / qubits).
    RNG order: the graph first, then ``theta[B][p][2]``.
    """
    rng = np.random.default_rng(seed)
    if edges is None:
        edges = random_regular3_graph(n, rng)
    gates = []
    for l in range(p):
        for (u, v) in edges:
            gates.append((RZZ, u, v, 2 * l, 0.0))
        for q in range(n):
            gates.append((RX, q, -1, 2 * l + 1, 0.0))
    theta = rng.uniform(0.0, math.pi, size=(B, p, 2)).reshape(B, 2 * p)
    terms = [(1.0, (u, v), "ZZ") for (u, v) in edges]
    return Problem(n=n, gates=gates, n_params=2 * p, terms=terms,
                   theta=np.ascontiguousarray(theta),
                   name=name or f"qaoa3reg_n{n}_p{p}",
                   meta={"p": p, "edges": edges, "layout": "dense"})


# ---------------------------------------------------------------------------
# The five workloads the benchmark and parity tests are built around.
# ---------------------------------------------------------------------------

def tfim_n8_L2(seed: int = 0) -> Problem:
    """n=8, L=2, J=h=1, one parameter set (forward energy)."""
    return tfim_problem(8, 2, 1, seed, name="tfim_n8_L2_B1")


def tfim_n20_L6_B64(seed: int = 1, B: int = 64) -> Problem:
    """n=20, L=6, J=1, h_i ~ U[0.5,1.5], 64 parameter sets (energy + gradient)."""
    return tfim_problem(20, 6, B, seed, h_range=(0.5, 1.5), name=f"tfim_n20_L6_B{B}")


def qaoa_n28_p4(seed: int = 2, n: int = 28, B: int = 1) -> Problem:
    """n=28 3-regular graph (42 edges), p=4, dense statevector workload."""
    return qaoa_problem(n, 4, B, seed, name=f"qaoa3reg_n{n}_p4")


def tfim_n500_L4_B256(seed: int = 3, B: int = 256) -> Problem:
    """n=500, L=4, J=h=1, 256 parameter sets (energy + gradient)."""
    return tfim_problem(500, 4, B, seed, name=f"tfim_n500_L4_B{B}")


@dataclass
class Request:
    t_arrival: float       # seconds from the start of the stream
    problem: Problem       # B = 1
    want_grad: bool


def serving_stream(count: int, rate: float, seed: int = 4,
                   n_range=(16, 400), L_range=(2, 8), grad_frac=0.3) -> list:
    """Poisson request stream: exponential inter-arrivals at ``rate``/s, then per
    request ``n ~ U[n_range]``, ``L ~ U[L_range]`` (inclusive integers), the mode
    (energy+gradient with probability ``grad_frac``) and the request's own seed."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps) - gaps[0]
    ns = rng.integers(n_range[0], n_range[1] + 1, size=count)
    Ls = rng.integers(L_range[0], L_range[1] + 1, size=count)
    grads = rng.random(size=count) < grad_frac
    seeds = rng.integers(0, 2**31 - 1, size=count)
    out = []
    for i in range(count):
        prob = tfim_problem(int(ns[i]), int(Ls[i]), 1, int(seeds[i]), h_range=(0.5, 1.5),
                            name=f"req{i}")
        out.append(Request(float(t[i]), prob, bool(grads[i])))
    return out


def random_local_problem(n: int, L: int, B: int, seed: int, kinds=("RY", "RX"),
                         with_rzz: bool = True) -> Problem:
    """A layered nearest-neighbour circuit with mixed gate kinds, used to widen
    parity coverage beyond the brick-wall: per layer a rotation (RX or RY, drawn
    per qubit) on every qubit, RZ on a random subset, then nearest-neighbour
    CZ or RZZ on random pairs. Hamiltonian: random one- and two-site Pauli strings."""
    rng = np.random.default_rng(seed)
    kind_ids = {"RX": RX, "RY": RY}
    gates = []
    P = 0
    for _ in range(L):
        for q in range(n):
            k = kind_ids[kinds[int(rng.integers(len(kinds)))]]
            gates.append((k, q, -1, P, 0.0))
            P += 1
        for q in range(n):
            if rng.random() < 0.6:
                gates.append((RZ, q, -1, P, 0.0))
                P += 1
        for q in range(n - 1):
            r = rng.random()
            if r < 0.4:
                gates.append((CZ, q, q + 1, -1, 0.0))
            elif r < 0.7 and with_rzz:
                gates.append((RZZ, q, q + 1, P, 0.0))
                P += 1
    terms = []
    letters = "XYZ"
    for i in range(n):
        terms.append((float(rng.uniform(-1, 1)), (i,), letters[int(rng.integers(3))]))
    for i in range(n - 1):
        terms.append((float(rng.uniform(-1, 1)), (i, i + 1),
                      letters[int(rng.integers(3))] + letters[int(rng.integers(3))]))
    theta = rng.uniform(0.0, 2.0 * math.pi, size=(B, P))
    return Problem(n=n, gates=gates, n_params=P, terms=terms, theta=theta,
                   name=f"local_n{n}_L{L}", meta={"L": L, "layout": "local"})


def random_nonlocal_problem(n: int, L: int, B: int, seed: int) -> Problem:
    """A layered circuit with two-qubit gates between arbitrary qubit pairs (dense path):
    per layer RX or RY (drawn per qubit) on every qubit, RZ on a random half, then n
    two-qubit gates on random pairs, each CZ or RZZ with its own angle; one in five RZ/RZZ
    reuses the previous parameter (shared angles) and one RZ per layer has a fixed angle.
    Hamiltonian: 2n random Pauli strings of 1-3 sites over X, Y, Z, coefficients U(-1, 1)."""
    rng = np.random.default_rng(seed)
    gates, P = [], 0
    for _ in range(L):
        for q in range(n):
            gates.append((RY if rng.random() < 0.5 else RX, q, -1, P, 0.0))
            P += 1
        for q in range(n):
            if rng.random() < 0.5:
                if P > 0 and rng.random() < 0.2:
                    gates.append((RZ, q, -1, P - 1, 0.0))
                else:
                    gates.append((RZ, q, -1, P, 0.0))
                    P += 1
        gates.append((RZ, int(rng.integers(n)), -1, -1, float(rng.uniform(0, 2 * np.pi))))
        for _ in range(n if n > 1 else 0):
            u, v = (int(x) for x in rng.choice(n, 2, replace=False))
            if rng.random() < 0.5:
                gates.append((CZ, u, v, -1, 0.0))
            elif P > 0 and rng.random() < 0.2:
                gates.append((RZZ, u, v, P - 1, 0.0))
            else:
                gates.append((RZZ, u, v, P, 0.0))
                P += 1
    terms = []
    for _ in range(2 * n):
        k = int(rng.integers(1, min(3, n) + 1))
        sites = tuple(int(s) for s in rng.choice(n, k, replace=False))
        terms.append((float(rng.uniform(-1, 1)), sites, "".join("XYZ"[int(rng.integers(3))] for _ in sites)))
    theta = rng.uniform(0, 2 * np.pi, size=(B, P))
    return Problem(n=n, gates=gates, n_params=P, terms=terms, theta=theta, name=f"nonlocal_n{n}_L{L}")
