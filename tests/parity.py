"""Tolerances shared by the GPU parity tests.

Energy: |E - E_ref| <= tol * max(|E_ref|, 1) with tol = 1e-5 for the FP32 state path and
1e-12 for the FP64 reference mode. Gradient: ||g - g_ref||_inf <= 1e-4 * max(1, ||g_ref||_inf)
(1e-11 in FP64 mode). The raw errors are returned so tests can print them.
"""
import numpy as np

E_TOL = {0: 1e-5, 1: 1e-5, 2: 1e-12}
G_TOL = {0: 1e-4, 1: 1e-4, 2: 1e-11}


def energy_err(E, Eref):
    E, Eref = np.asarray(E, dtype=np.float64), np.asarray(Eref, dtype=np.float64)
    return float(np.max(np.abs(E - Eref) / np.maximum(np.abs(Eref), 1.0)))


def grad_err(g, gref):
    g, gref = np.asarray(g, dtype=np.float64), np.asarray(gref, dtype=np.float64)
    return float(np.max(np.abs(g - gref)) / max(1.0, float(np.max(np.abs(gref)))))


def check_energy(E, Eref, prec=0):
    err = energy_err(E, Eref)
    assert err <= E_TOL[prec], f"energy error {err:.3e} > {E_TOL[prec]:.0e}"
    return err


def check_grad(g, gref, prec=0):
    err = grad_err(g, gref)
    assert err <= G_TOL[prec], f"gradient error {err:.3e} > {G_TOL[prec]:.0e}"
    return err
