"""Post-processing of the measured observables (Sec. 2.2).

These act on the FP64 results the library returns (Polyakov loop means,
correlator sums); none of them touches the lattice.

* renormalised Polyakov loop  <L^r> = Z(g^2)^Nt <L>,  Z = exp(A g^2 + B g^4)
  with the fit values the paper prints, A = 0.0637(18), B = 0.0731(16),
  valid for g^2 < 1.3 (Sec. 2.2, Eq. 2); g^2 = 4 / beta for SU(2).
* colour-averaged free energy from the correlator (Sec. 2.2, Eq. 3):
  exp(-F/T + c) = 1/4 <Tr L(y) Tr L^+(x)> = C(r) in the library's
  normalisation (L = 1/2 Tr), shifted by -T ln 4; in lattice units
  (a = 1) T = 1 / Nt.  The unknown constant c is dropped.
* the fit F(r) = a0 - a1 / r + sigma r that gives the string tension, and
  the two sigma(T) forms the paper fits.
"""
from __future__ import annotations

import numpy as np

A_PAPER = 0.0637   # +- 0.0018
B_PAPER = 0.0731   # +- 0.0016
G2_MAX = 1.3       # range of the paper's fit


def g2_of_beta(beta):
    """Bare coupling of the Wilson action S = beta sum (1 - 1/2 Re Tr U_P)."""
    return 4.0 / np.asarray(beta, dtype=np.float64)


def renormalisation_constant(beta, A: float = A_PAPER, B: float = B_PAPER):
    g2 = g2_of_beta(beta)
    return np.exp(A * g2 + B * g2 ** 2)


def renormalised_polyakov(L, beta, Nt: int, A: float = A_PAPER, B: float = B_PAPER,
                          check_range: bool = True):
    """<L^r> = Z(g^2)^Nt <L> (Sec. 2.2, Eq. 2)."""
    g2 = g2_of_beta(beta)
    if check_range and np.any(g2 >= G2_MAX):
        raise ValueError("the printed Z(g^2) fit holds for g^2 < 1.3 (beta > 3.08)")
    return renormalisation_constant(beta, A, B) ** Nt * np.asarray(L, dtype=np.float64)


def free_energy(C, Nt: int):
    """F_avg(r) in lattice units from C(r) = <L(x) L(x+r)> (Sec. 2.2, Eq. 3):
    F = -T ln C(r) - T ln 4 with T = 1/Nt; C(r) must be positive."""
    C = np.asarray(C, dtype=np.float64)
    if np.any(C <= 0):
        raise ValueError("the correlator must be positive to take its logarithm")
    T = 1.0 / Nt
    return -T * np.log(C) - T * np.log(4.0)


def fit_string_tension(r, F, err=None):
    """Weighted least squares of F(r) = a0 - a1 / r + sigma r.
    Returns ((a0, a1, sigma), covariance)."""
    r = np.asarray(r, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64)
    w = np.ones_like(F) if err is None else 1.0 / np.asarray(err, dtype=np.float64) ** 2
    X = np.stack([np.ones_like(r), -1.0 / r, r], axis=1)
    XtW = X.T * w
    cov = np.linalg.inv(XtW @ X)
    coef = cov @ (XtW @ F)
    if err is None:  # scale by the residual variance
        res = F - X @ coef
        dof = max(len(F) - 3, 1)
        cov = cov * float(res @ res) / dof
    return tuple(coef), cov


def sigma_ansatz_sqrt(t, a, b):
    """sigma(T) = a sqrt(1 - b (T/T_c)^2), t = T/T_c (Sec. 2.2)."""
    return a * np.sqrt(1.0 - b * np.asarray(t, dtype=np.float64) ** 2)


def sigma_ansatz_ising(dT, a, b, nu: float = 0.63):
    """sigma(T) = a (T_c - T)^nu [1 + b sqrt(T_c - T)], dT = T_c - T, with the
    3D Ising exponent nu = 0.63 (Sec. 2.2)."""
    dT = np.asarray(dT, dtype=np.float64)
    return a * dT ** nu * (1.0 + b * np.sqrt(dT))
