"""Write the stored expected values under tests/golden/ (calls only the CPU oracle).

Each fixture stores its inputs (angles, coefficients, gate list) next to the
oracle's outputs, so a parity test reads both from the file and depends on no
random-number stream at test time.

    python tests/golden/make_golden.py            # the small fixtures
    python tests/golden/make_golden.py --large    # also the n=28 QAOA fixture (about 8 GiB of
                                                  # host memory, minutes on a few cores)
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import dense  # noqa: E402
from paper_2112_10239_gb300 import workloads as W  # noqa: E402


def dump(name, prob, cite):
    th = prob.theta[0]
    E, et = dense.energy_terms(prob.n, prob.gates, prob.terms, th)
    Eg, g = dense.grad_adjoint(prob.n, prob.gates, prob.terms, th, prob.n_params)
    out = {
        "cite": cite,
        "written_by": "tests/golden/make_golden.py (CPU oracle, complex128)",
        "n": prob.n,
        "n_params": prob.n_params,
        "gates": [list(g_) for g_ in prob.gates],
        "terms": [[c, list(s), l] for (c, s, l) in prob.terms],
        "theta": [float(x) for x in th],
        "energy": E,
        "term_values": [float(x) for x in et],
        "grad": [float(x) for x in g],
    }
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(out, f, indent=1)
    print(name, E)


def dump_grad_only(name, prob, cite):
    """Energy and full gradient from the oracle's adjoint sweep (one forward, one backward
    pass over the 2^n complex128 state); for states too large to also store term values."""
    th = prob.theta[0]
    E, g = dense.grad_adjoint(prob.n, prob.gates, prob.terms, th, prob.n_params)
    out = {
        "cite": cite,
        "written_by": "tests/golden/make_golden.py --large (CPU oracle, complex128)",
        "n": prob.n,
        "n_params": prob.n_params,
        "gates": [list(g_) for g_ in prob.gates],
        "terms": [[c, list(s), l] for (c, s, l) in prob.terms],
        "theta": [float(x) for x in th],
        "energy": E,
        "grad": [float(x) for x in g],
    }
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(out, f, indent=1)
    print(name, E)


if __name__ == "__main__":
    dump("tfim_n8_L2.json", W.tfim_n8_L2(seed=0),
         "Transverse-field Ising expectation value and its full gradient "
         "(TensorLy-Quantum Sec. 3); n=8, L=2 brick-wall, J=h=1")
    dump("local_mixed_n7_L3.json", W.random_local_problem(7, 3, 1, seed=21),
         "Expectation value of a Pauli-sum operator for a circuit of pre-defined gates "
         "(TensorLy-Quantum Sec. 2 and Sec. 3); mixed RX/RY/RZ/RZZ/CZ nearest-neighbour circuit")
    if "--large" in sys.argv:
        dump_grad_only("qaoa_n28_p4.json", W.qaoa_n28_p4(seed=2),
                       "Expectation value and full gradient for an all-to-all circuit on the dense "
                       "statevector (TensorLy-Quantum Sec. 1 vector representation, Sec. 3 expectation "
                       "and gradient); QAOA p=4 on a seeded 3-regular graph, n=28, 42 edges")
