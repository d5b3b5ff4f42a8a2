"""Pins for the CPU oracle: results the mathematics fixes independently of the oracle.

Each test is chosen so that a plausible slip in the oracle (a wrong sign in a gate,
a transposed rotation, a dropped CZ, a wrong Pauli phase, a wrong bit order, a
wrong adjoint sign, a light-cone window that drops a gate) fails at least one of
them. Nothing here touches the CUDA path.
"""
import math

import numpy as np
import pytest

from oracle import dense, ed, windows
from paper_2112_10239_gb300 import workloads as W

RX, RY, RZ, RZZ, CZ = W.RX, W.RY, W.RZ, W.RZZ, W.CZ
HALF_PI = math.pi / 2


def _product_gates(n):
    return [(RY, q, -1, q, 0.0) for q in range(n)] + [(RZ, q, -1, n + q, 0.0) for q in range(n)]


@pytest.mark.parametrize("seed", range(4))
def test_product_state_closed_forms(seed):
    # <Z_i> = cos a_i, <X_i> = sin a_i cos b_i, <Y_i> = sin a_i sin b_i,
    # <Z_i Z_j> = cos a_i cos a_j for RZ(b) RY(a) |0> on every qubit.
    rng = np.random.default_rng(seed)
    n = 5
    a, b = rng.uniform(0, 2 * math.pi, n), rng.uniform(0, 2 * math.pi, n)
    th = np.concatenate([a, b])
    psi = dense.statevector(n, _product_gates(n), th)
    for q in range(n):
        assert dense.pauli_expectation(n, psi, (q,), "Z") == pytest.approx(math.cos(a[q]), abs=1e-13)
        assert dense.pauli_expectation(n, psi, (q,), "X") == pytest.approx(
            math.sin(a[q]) * math.cos(b[q]), abs=1e-13)
        assert dense.pauli_expectation(n, psi, (q,), "Y") == pytest.approx(
            math.sin(a[q]) * math.sin(b[q]), abs=1e-13)
    for i in range(n):
        for j in range(i + 1, n):
            assert dense.pauli_expectation(n, psi, (i, j), "ZZ") == pytest.approx(
                math.cos(a[i]) * math.cos(a[j]), abs=1e-13)


def test_rx_closed_form():
    # RX(a)|0>: <Z> = cos a, <Y> = -sin a, <X> = 0.
    for a in (0.3, 1.7, 4.1):
        psi = dense.statevector(1, [(RX, 0, -1, -1, a)], [0.0])
        assert dense.pauli_expectation(1, psi, (0,), "Z") == pytest.approx(math.cos(a), abs=1e-14)
        assert dense.pauli_expectation(1, psi, (0,), "Y") == pytest.approx(-math.sin(a), abs=1e-14)
        assert dense.pauli_expectation(1, psi, (0,), "X") == pytest.approx(0.0, abs=1e-14)


def test_rzz_closed_form():
    # RZZ(g) on RY(a0)|0> x |0>: with qubit 1 in |0>, RZZ acts on qubit 0 as RZ(g),
    # so <X_0> = sin a0 cos g, <Y_0> = sin a0 sin g and <Z_0> = cos a0.
    for a0, g in ((0.9, 0.4), (2.2, 1.3)):
        gates = [(RY, 0, -1, -1, a0), (RZZ, 0, 1, -1, g)]
        psi = dense.statevector(2, gates, [0.0])
        assert dense.pauli_expectation(2, psi, (0,), "X") == pytest.approx(math.sin(a0) * math.cos(g), abs=1e-14)
        assert dense.pauli_expectation(2, psi, (0,), "Y") == pytest.approx(math.sin(a0) * math.sin(g), abs=1e-14)
        assert dense.pauli_expectation(2, psi, (0,), "Z") == pytest.approx(math.cos(a0), abs=1e-14)


@pytest.mark.parametrize("n", [2, 5, 6, 7])
def test_layer1_brickwall_closed_form(n):
    # One RY/RZ + CZ brick-wall layer: CZ X_i CZ = X_i Z_j gives
    # E = J sum_i cos a_i cos a_{i+1} + sum_i h_i sin a_i cos b_i prod_{j in {i-1,i+1}} cos a_j.
    p = W.tfim_problem(n, 1, 3, seed=10 + n, h_range=(0.5, 1.5))
    h = p.meta["h"]
    for th in p.theta:
        a, b = th[:n], th[n:2 * n]
        E = sum(math.cos(a[i]) * math.cos(a[i + 1]) for i in range(n - 1))
        for i in range(n):
            nb = [math.cos(a[j]) for j in (i - 1, i + 1) if 0 <= j < n]
            E += h[i] * math.sin(a[i]) * math.cos(b[i]) * float(np.prod(nb))
        assert dense.energy(n, p.gates, p.terms, th) == pytest.approx(E, abs=1e-13)


def test_bell_correlators():
    # RY(pi/2) x RY(pi/2), CZ, RY(-pi/2) on qubit 1 gives (|00> - |11>)/sqrt 2.
    g = [(RY, 0, -1, -1, HALF_PI), (RY, 1, -1, -1, HALF_PI), (CZ, 0, 1, -1, 0.0),
         (RY, 1, -1, -1, -HALF_PI)]
    psi = dense.statevector(2, g, [0.0])
    r = 1 / math.sqrt(2)
    assert np.allclose(psi, [r, 0, 0, -r], atol=1e-15)
    assert dense.pauli_expectation(2, psi, (0, 1), "ZZ") == pytest.approx(1.0, abs=1e-14)
    assert dense.pauli_expectation(2, psi, (0, 1), "XX") == pytest.approx(-1.0, abs=1e-14)
    assert dense.pauli_expectation(2, psi, (0, 1), "YY") == pytest.approx(1.0, abs=1e-14)
    assert dense.pauli_expectation(2, psi, (0, 1), "XY") == pytest.approx(0.0, abs=1e-14)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 8])
def test_ghz_ladder(n):
    # RY(pi/2) on q0, then RY(pi/2)_t CZ(t-1,t) RY(-pi/2)_t: each rung maps the
    # target to -|1> when the control is 1, so psi = (|0..0> + (-1)^(n-1) |1..1>)/sqrt 2.
    g = [(RY, 0, -1, -1, HALF_PI)]
    for t in range(1, n):
        g += [(RY, t, -1, -1, HALF_PI), (CZ, t - 1, t, -1, 0.0), (RY, t, -1, -1, -HALF_PI)]
    psi = dense.statevector(n, g, [0.0])
    want = np.zeros(2 ** n)
    want[0] = 1 / math.sqrt(2)
    want[-1] = (-1) ** (n - 1) / math.sqrt(2)
    assert np.allclose(psi, want, atol=1e-14)
    for i in range(n):
        for j in range(i + 1, n):
            assert dense.pauli_expectation(n, psi, (i, j), "ZZ") == pytest.approx(1.0, abs=1e-14)
    assert dense.pauli_expectation(n, psi, tuple(range(n)), "X" * n) == pytest.approx(
        (-1) ** (n - 1), abs=1e-14)


@pytest.mark.parametrize("seed", range(3))
def test_norm_preserved(seed):
    p = W.random_local_problem(9, 3, 1, seed)
    psi = dense.statevector(p.n, p.gates, p.theta[0])
    assert np.linalg.norm(psi) == pytest.approx(1.0, abs=1e-14)


@pytest.mark.parametrize("seed", range(3))
def test_exact_diagonalisation(seed):
    # psi^dag H psi with an explicit matrix equals the oracle's Pauli-sum energy,
    # and the variational bound E >= lambda_min(H) holds.
    p = W.tfim_problem(8, 2, 2, seed, h_range=(0.5, 1.5))
    H = ed.hamiltonian_matrix(p.n, p.terms)
    lam0 = ed.ground_energy(H)
    for th in p.theta:
        psi = dense.statevector(p.n, p.gates, th)
        E = dense.energy(p.n, p.gates, p.terms, th)
        assert ed.expectation(H, psi) == pytest.approx(E, abs=1e-12)
        assert E >= lam0 - 1e-12
    q = W.random_local_problem(6, 2, 1, seed)
    H = ed.hamiltonian_matrix(q.n, q.terms)
    psi = dense.statevector(q.n, q.gates, q.theta[0])
    assert ed.expectation(H, psi) == pytest.approx(dense.energy(q.n, q.gates, q.terms, q.theta[0]), abs=1e-12)


def test_exact_diagonalisation_tfim_ground_state():
    # Independent of any circuit: H = Z Z + X_0 + X_1 (n=2) splits into the block
    # [[1, 2], [2, -1]] on span{(|00>+|11>)/sqrt2, (|01>+|10>)/sqrt2} plus the
    # eigenvalues 1 and -1, so its ground energy is -sqrt(5).
    H = ed.hamiltonian_matrix(2, W.tfim_terms(2, 1.0, 1.0))
    assert ed.ground_energy(H) == pytest.approx(-math.sqrt(5.0), abs=1e-12)


@pytest.mark.parametrize("seed", range(2))
def test_adjoint_equals_parameter_shift(seed):
    p = W.tfim_problem(6, 2, 1, seed, h_range=(0.5, 1.5))
    E, g = dense.grad_adjoint(p.n, p.gates, p.terms, p.theta[0], p.n_params)
    ps = dense.grad_param_shift(p.n, p.gates, p.terms, p.theta[0], range(p.n_params))
    assert E == pytest.approx(dense.energy(p.n, p.gates, p.terms, p.theta[0]), abs=1e-13)
    assert np.max(np.abs(g - ps)) < 1e-12


def test_adjoint_mixed_kinds_equals_parameter_shift():
    # RX, RY, RZ, RZZ and every Pauli letter (one rotation per parameter).
    p = W.random_local_problem(6, 2, 1, seed=11)
    E, g = dense.grad_adjoint(p.n, p.gates, p.terms, p.theta[0], p.n_params)
    ps = dense.grad_param_shift(p.n, p.gates, p.terms, p.theta[0], range(p.n_params))
    assert np.max(np.abs(g - ps)) < 1e-12


def test_adjoint_shared_parameter_sums_gates():
    # A parameter on several gates (QAOA's shared gamma/beta) gets the sum of the
    # per-gate derivatives; check against central differences (O(h^2) = 1e-6 at h=1e-3).
    p = W.qaoa_problem(8, 2, 1, seed=5)
    E, g = dense.grad_adjoint(p.n, p.gates, p.terms, p.theta[0], p.n_params)
    fd = dense.grad_fd(p.n, p.gates, p.terms, p.theta[0], range(p.n_params), h=1e-3)
    assert np.max(np.abs(g - fd)) < 5e-6 * max(1.0, np.max(np.abs(g)))
    fd2 = dense.grad_fd(p.n, p.gates, p.terms, p.theta[0], range(p.n_params), h=2e-3)
    # Richardson: the FD error scales as h^2.
    e1, e2 = np.max(np.abs(fd - g)), np.max(np.abs(fd2 - g))
    assert e2 > 3.0 * e1


def test_fd_agrees_at_tfim_n8():
    p = W.tfim_n8_L2()
    E, g = dense.grad_adjoint(p.n, p.gates, p.terms, p.theta[0], p.n_params)
    fd = dense.grad_fd(p.n, p.gates, p.terms, p.theta[0], range(p.n_params), h=1e-3)
    assert np.max(np.abs(g - fd)) < 1e-5


def test_last_layer_rz_gradient_vanishes_for_z_terms():
    # The last RZ layer commutes with Z-only terms; with h = 0 dE/db_L = 0 exactly.
    n, L = 6, 3
    p = W.tfim_problem(n, L, 1, seed=4)
    terms = W.tfim_terms(n, 1.0, 0.0)
    _, g = dense.grad_adjoint(n, p.gates, terms, p.theta[0], p.n_params)
    bL = [(L - 1) * 2 * n + n + q for q in range(n)]
    assert np.max(np.abs(g[bL])) < 1e-14
    # ... and it does not vanish with the transverse field on.
    _, g = dense.grad_adjoint(n, p.gates, p.terms, p.theta[0], p.n_params)
    assert np.max(np.abs(g[bL])) > 1e-3


@pytest.mark.parametrize("n,L", [(12, 2), (14, 3), (16, 4)])
def test_cone_windows_equal_full_chain(n, L):
    p = W.tfim_problem(n, L, 1, seed=n + L, h_range=(0.5, 1.5))
    cc = windows.ConeCache(p.gates, p.terms)
    Ew, et_w = cc.energy_terms(p.theta[0])
    Ef, et_f = dense.energy_terms(p.n, p.gates, p.terms, p.theta[0])
    assert np.max(np.abs(et_w - et_f)) < 1e-12
    Eg, g = cc.grad(p.theta[0], p.n_params)
    Egf, gf = dense.grad_adjoint(p.n, p.gates, p.terms, p.theta[0], p.n_params)
    assert Eg == pytest.approx(Egf, abs=1e-12)
    assert np.max(np.abs(g - gf)) < 1e-12


def test_too_narrow_window_is_wrong():
    # Negative control for the window test: drop the outermost qubits of one interior
    # X term's cone (simulate only gates fully inside [lo+1, hi-1]) and the value
    # changes, so the window comparison above has teeth.
    n, L = 14, 3
    p = W.tfim_problem(n, L, 1, seed=1, h_range=(0.5, 1.5))
    i = 7
    exact = dense.pauli_expectation(n, dense.statevector(n, p.gates, p.theta[0]), (i,), "X")
    lo, hi = i - L, i + L   # exact cone of X_i: 2L+1 sites
    for (a, b) in ((lo, hi), (lo + 1, hi), (lo, hi - 1)):
        sub = [(k, q0 - a, (q1 - a) if q1 >= 0 else -1, pp, ang) for (k, q0, q1, pp, ang) in p.gates
               if a <= q0 <= b and (q1 < 0 or a <= q1 <= b)]
        w = b - a + 1
        val = dense.energy(w, sub, [(1.0, (i - a,), "X")], p.theta[0])
        if (a, b) == (lo, hi):
            assert val == pytest.approx(exact, abs=1e-12)
        else:
            assert abs(val - exact) > 1e-6


@pytest.mark.parametrize("seed", range(2))
def test_qaoa_closed_forms(seed):
    n = 10
    p = W.qaoa_problem(n, 1, 3, seed)
    m = len(p.meta["edges"])
    for th in p.theta:
        # p = 1 from |0..0>: RZZ is a global phase, so E = |edges| cos^2 beta.
        assert dense.energy(n, p.gates, p.terms, th) == pytest.approx(m * math.cos(th[1]) ** 2, abs=1e-12)
        # and its gradient: dE/dgamma_1 = 0 (a global phase), dE/dbeta_1 = -|edges| sin(2 beta)
        _, g = dense.grad_adjoint(n, p.gates, p.terms, th, p.n_params)
        assert g[0] == pytest.approx(0.0, abs=1e-12)
        assert g[1] == pytest.approx(-m * math.sin(2 * th[1]), abs=1e-12)
    q = W.qaoa_problem(n, 3, 1, seed)
    th = q.theta[0].copy()
    th[1::2] = 0.0   # every beta = 0: the state stays |0..0> up to phase
    assert dense.energy(n, q.gates, q.terms, th) == pytest.approx(float(m), abs=1e-12)


def test_qaoa_energy_is_cut_function():
    # E = sum_x |psi_x|^2 C(x) with C(x) = sum_e z_u z_v, and C(x) = C(~x).
    n = 10
    p = W.qaoa_problem(n, 2, 1, seed=3)
    psi = dense.statevector(n, p.gates, p.theta[0])
    x = np.arange(2 ** n)
    C = np.zeros(2 ** n)
    for (u, v) in p.meta["edges"]:
        C += (1 - 2 * ((x >> u) & 1)) * (1 - 2 * ((x >> v) & 1))
    assert np.allclose(C, C[::-1])
    assert float(np.sum(np.abs(psi) ** 2 * C)) == pytest.approx(
        dense.energy(n, p.gates, p.terms, p.theta[0]), abs=1e-12)


def test_translation_invariance_interior_terms():
    # Uniform angles and field: interior terms of the same kind are equal.
    n, L = 16, 2
    p = W.tfim_problem(n, L, 1, seed=0)
    th = np.zeros(p.n_params)
    for l in range(L):
        th[l * 2 * n: l * 2 * n + n] = 0.7 + l
        th[l * 2 * n + n: (l + 1) * 2 * n] = 1.9 - l
    _, et = dense.energy_terms(n, p.gates, p.terms, th)
    zz, xx = et[: n - 1], et[n - 1:]
    # sites far from both ends, same parity (the brick-wall has period 2)
    assert abs(zz[6] - zz[8]) < 1e-13 and abs(zz[7] - zz[9]) < 1e-13
    assert abs(xx[6] - xx[8]) < 1e-13 and abs(xx[7] - xx[9]) < 1e-13


def test_relabel_invariance():
    # Mirroring the chain (q -> n-1-q) in both circuit and Hamiltonian keeps E.
    n = 7
    p = W.random_local_problem(n, 2, 1, seed=2)
    mg = [(k, n - 1 - q0, (n - 1 - q1) if q1 >= 0 else -1, pp, a) for (k, q0, q1, pp, a) in p.gates]
    mt = [(c, tuple(n - 1 - s for s in sites), l) for (c, sites, l) in p.terms]
    assert dense.energy(n, mg, mt, p.theta[0]) == pytest.approx(
        dense.energy(n, p.gates, p.terms, p.theta[0]), abs=1e-13)


# ---- partial trace (reduced density operators of pure states) ---------------------------

_PAULI = {"I": np.eye(2), "X": np.array([[0, 1], [1, 0]], dtype=complex),
          "Y": np.array([[0, -1j], [1j, 0]]), "Z": np.diag([1.0, -1.0]).astype(complex)}


def _kron_sites(mats_by_site, keep):
    """Operator on the kept qubits with bit t of the index = qubit keep[t]."""
    out = np.eye(1, dtype=complex)
    for q in sorted(keep, reverse=True):   # most significant factor first
        out = np.kron(out, mats_by_site[q])
    return out


@pytest.mark.parametrize("seed", range(3))
def test_partial_trace_product_state(seed):
    # |psi> = prod_q RZ(b_q) RY(a_q) |0>: every reduced state is the product of the
    # single-qubit states phi_q = (cos(a/2) e^{-ib/2}, sin(a/2) e^{ib/2}).
    from oracle import density
    rng = np.random.default_rng(seed)
    n = 6
    a, b = rng.uniform(0, 2 * np.pi, n), rng.uniform(0, 2 * np.pi, n)
    gates = [(W.RY, q, -1, q, 0.0) for q in range(n)] + [(W.RZ, q, -1, n + q, 0.0) for q in range(n)]
    psi = dense.statevector(n, gates, np.concatenate([a, b]))
    phi = {q: np.array([math.cos(a[q] / 2) * np.exp(-0.5j * b[q]), math.sin(a[q] / 2) * np.exp(0.5j * b[q])])
           for q in range(n)}
    for keep in ([0], [2], [1, 4], [0, 3, 5], list(range(n))):
        rho = density.reduced_density(psi, n, keep)
        want = _kron_sites({q: np.outer(phi[q], phi[q].conj()) for q in keep}, keep)
        assert np.max(np.abs(rho - want)) < 1e-13


def test_partial_trace_bell_and_ghz():
    from oracle import density
    half = math.pi / 2
    bell = dense.statevector(2, [(W.RY, 0, -1, -1, half), (W.RY, 1, -1, -1, half), (W.CZ, 0, 1, -1, 0.0),
                                 (W.RY, 1, -1, -1, -half)], [0.0])
    for keep in ([0], [1]):
        assert np.max(np.abs(density.reduced_density(bell, 2, keep) - np.eye(2) / 2)) < 1e-14
    n = 5
    gates = [(W.RY, 0, -1, -1, half)]
    for t in range(1, n):
        gates += [(W.RY, t, -1, -1, half), (W.CZ, t - 1, t, -1, 0.0), (W.RY, t, -1, -1, -half)]
    ghz = dense.statevector(n, gates, [0.0])
    rho = density.reduced_density(ghz, n, [3, 0])
    want = np.zeros((4, 4))
    want[0, 0] = want[3, 3] = 0.5
    assert np.max(np.abs(rho - want)) < 1e-14


@pytest.mark.parametrize("seed", range(4))
def test_partial_trace_properties_and_pauli_expectations(seed):
    # random entangled state: rho_A is Hermitian, PSD, of unit trace, and Tr(rho_A P_A)
    # equals <psi|P_A|psi> evaluated on the full state by the C oracle
    from oracle import density
    rng = np.random.default_rng(40 + seed)
    prob = W.random_nonlocal_problem(7, 2, 1, seed=seed)
    psi = dense.statevector(prob.n, prob.gates, prob.theta[0])
    for _ in range(4):
        m = int(rng.integers(1, prob.n + 1))
        keep = sorted(int(q) for q in rng.choice(prob.n, m, replace=False))
        rho = density.reduced_density(psi, prob.n, keep)
        assert abs(np.trace(rho) - 1) < 1e-13
        assert np.max(np.abs(rho - rho.conj().T)) < 1e-14
        assert np.min(np.linalg.eigvalsh(rho)) > -1e-13
        for _ in range(3):
            k = int(rng.integers(1, m + 1))
            sites = [int(q) for q in rng.choice(keep, k, replace=False)]
            letters = "".join("XYZ"[int(rng.integers(3))] for _ in sites)
            P = _kron_sites({q: _PAULI[letters[sites.index(q)]] if q in sites else _PAULI["I"] for q in keep}, keep)
            want = dense.pauli_expectation(prob.n, psi, sites, letters)
            assert abs(np.trace(rho @ P).real - want) < 1e-13
    # keeping every qubit gives the pure density operator itself
    full = density.reduced_density(psi, prob.n, range(prob.n))
    assert np.max(np.abs(full - np.outer(psi, psi.conj()))) < 1e-15


@pytest.mark.parametrize("seed,top_kind,pair_kind", [(0, RY, CZ), (1, RX, RZZ), (2, RY, RZZ), (3, RX, CZ)])
def test_window_branch_decomposition(seed, top_kind, pair_kind):
    # The CUDA cone kernel splits a window whose top qubit t carries gates of the first layer
    # only and no measured term into the branches t = 0 and t = 1. Check the mathematics it
    # relies on with the oracle alone: with p_h the weight |f_t(h)|^2 of the top qubit's
    # first-layer rotation (cos^2 a/2, sin^2 a/2) and E_h the energy of the (W-1)-qubit circuit
    # whose pair gate (t-1, t) is replaced by its action at t = h (CZ: Z on t-1 for h = 1;
    # RZZ(g): RZ((-1)^h g) on t-1), E = p_0 E_0 + p_1 E_1, and dE/da = sin(a)/2 (E_1 - E_0).
    rng = np.random.default_rng(seed)
    n, t = 9, 8
    gates, P = [], 0
    for q in range(n):   # first layer: rotations on every qubit, RZ, pairs (including (t-1, t))
        gates.append((top_kind if q == t else int(rng.choice([RX, RY])), q, -1, P, 0.0))
        P += 1
    for q in range(n):
        gates.append((RZ, q, -1, P, 0.0))
        P += 1
    for q in range(n - 1):
        kind = pair_kind if q == t - 1 else int(rng.choice([CZ, RZZ]))
        gates.append((kind, q, q + 1, P if kind == RZZ else -1, 0.0))
        P += kind == RZZ
    rest = []
    for _ in range(3):   # later layers never touch t
        for q in range(t):
            rest.append((int(rng.choice([RX, RY])), q, -1, P, 0.0))
            P += 1
        for q in range(t - 1):
            rest.append((RZZ, q, q + 1, P, 0.0))
            P += 1
    terms = [(float(rng.uniform(-1, 1)), (q,), "XYZ"[int(rng.integers(3))]) for q in range(t)]
    terms += [(float(rng.uniform(-1, 1)), (q, q + 1), "ZZ") for q in range(t - 1)]
    theta = rng.uniform(0, 2 * math.pi, size=P)
    full = gates + rest
    E, g = dense.grad_adjoint(n, full, terms, theta, P)
    a_idx = next(G[3] for G in gates if G[1] == t and G[0] in (RX, RY))
    a = theta[a_idx]
    pair = next(G for G in gates if G[0] in (CZ, RZZ) and G[1] == t - 1)
    Eh = []
    for h in (0, 1):
        # the branch circuit on qubits 0..t-1: gates not touching t, the pair gate at t = h
        br = [G for G in gates if G[1] != t and not (G[0] in (CZ, RZZ) and G[2] == t)]
        if pair[0] == CZ:
            if h == 1:
                br.append((RZ, t - 1, -1, -1, math.pi))   # Z on t-1 up to a global phase
        else:
            br.append((RZ, t - 1, -1, -1, (-1) ** h * theta[pair[3]]))
        Eh.append(dense.energy(t, br + rest, terms, theta))
    p0, p1 = math.cos(a / 2) ** 2, math.sin(a / 2) ** 2
    assert abs(E - (p0 * Eh[0] + p1 * Eh[1])) <= 1e-12
    assert abs(g[a_idx] - 0.5 * math.sin(a) * (Eh[1] - Eh[0])) <= 1e-10


@pytest.mark.parametrize("pair", [(0, 1), (2, 1), (1, 2)])
def test_two_qubit_gates_split_into_site_products(pair):
    # The exact MPS route writes each two-qubit gate as a sum of two products of single-site
    # operators, the first factor on the lower qubit: CZ = sum_b |b><b| (x) Z^b and
    # RZZ(g) = cos(g/2) I (x) I - i sin(g/2) Z (x) Z. Check both sums against the oracle's own
    # gates on random entangled 3-qubit states, with the gate's qubits given in either order.
    rng = np.random.default_rng(11)
    n = 3
    prep, P = [], 0
    for _ in range(2):
        for q in range(n):
            prep += [(RY, q, -1, P, 0.0), (RZ, q, -1, P + 1, 0.0)]
            P += 2
        prep += [(RZZ, 0, 1, P, 0.0), (RZZ, 1, 2, P + 1, 0.0)]
        P += 2
    theta = rng.uniform(0, 2 * math.pi, size=P + 1)
    psi = dense.statevector(n, prep, theta)
    lo, hi = min(pair), max(pair)

    def on(ops, v):   # apply {qubit: 2x2} to a state (bit q of the index is qubit q)
        t = v.reshape((2,) * n)   # axis k is qubit n - 1 - k
        for q, M in ops.items():
            t = np.moveaxis(np.tensordot(M, t, axes=([1], [n - 1 - q])), 0, n - 1 - q)
        return t.reshape(-1)

    I2, Z = np.eye(2), np.diag([1.0, -1.0])
    proj = [np.diag([1.0, 0.0]), np.diag([0.0, 1.0])]
    cz = dense.statevector(n, prep + [(CZ, pair[0], pair[1], -1, 0.0)], theta)
    split = sum(on({lo: proj[b], hi: np.linalg.matrix_power(Z, b)}, psi) for b in (0, 1))
    assert np.max(np.abs(cz - split)) < 1e-13
    g = theta[P]
    rzz = dense.statevector(n, prep + [(RZZ, pair[0], pair[1], P, 0.0)], theta)
    split = math.cos(g / 2) * psi - 1j * math.sin(g / 2) * on({lo: Z, hi: Z}, psi)
    assert np.max(np.abs(rzz - split)) < 1e-13
