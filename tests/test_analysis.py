"""Post-processing of Sec. 2.2 against closed forms and the numbers the
paper prints (tests/golden/paper_constants.json)."""
import json
import os

import numpy as np
import pytest

from paper_1104_5432_gb300 import analysis as A

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def test_printed_constants_are_the_ones_used():
    z = GOLDEN["renormalisation_Z"]
    assert (A.A_PAPER, A.B_PAPER, A.G2_MAX) == (z["A"], z["B"], z["g2_max"])
    assert A.sigma_ansatz_ising.__defaults__ == (GOLDEN["sigma_fit_ising"]["nu"],)


def test_fits_recover_the_printed_sigma_parameters():
    """Synthetic sigma(T) on the paper's two printed curves, fitted with the
    same forms by least squares: the printed parameters come back."""
    from scipy.optimize import curve_fit
    t = np.linspace(0.7, 0.98, 15)            # T / T_c
    sq = GOLDEN["sigma_fit_sqrt"]
    y = A.sigma_ansatz_sqrt(t, sq["a"], sq["b"])
    (a, b), _ = curve_fit(A.sigma_ansatz_sqrt, t, y, p0=(0.5, 0.9), bounds=([0.1, 0.5], [2.0, 1.04]))
    assert (a, b) == pytest.approx((sq["a"], sq["b"]), rel=1e-6)
    isg = GOLDEN["sigma_fit_ising"]
    dT = 1.0 - t                              # T_c - T in units of T_c
    y = A.sigma_ansatz_ising(dT, isg["a"], isg["b"])
    (a, b), _ = curve_fit(lambda d, a, b: A.sigma_ansatz_ising(d, a, b), dT, y, p0=(1.0, 0.0))
    assert (a, b) == pytest.approx((isg["a"], isg["b"]), rel=1e-6)
    # both printed curves describe the same sigma(T) near T_c to ~10%
    mid = np.array([0.85, 0.9])
    r = A.sigma_ansatz_sqrt(mid, sq["a"], sq["b"]) / A.sigma_ansatz_ising(1 - mid, isg["a"], isg["b"])
    assert np.all(np.abs(r - 1) < 0.15), r


def test_renormalised_polyakov_closed_form():
    # beta = 4: g^2 = 1, Z = exp(A + B) with the printed A, B
    Z = np.exp(0.0637 + 0.0731)
    assert A.renormalisation_constant(4.0) == pytest.approx(Z, rel=1e-15)
    assert A.renormalised_polyakov(0.2, 4.0, Nt=4) == pytest.approx(0.2 * Z ** 4, rel=1e-14)
    # Z > 1 and grows with Nt: the renormalised loop exceeds the bare one
    Lr = A.renormalised_polyakov([0.1, 0.1], [5.0, 5.0], Nt=6)
    assert np.all(Lr > 0.1)
    with pytest.raises(ValueError):
        A.renormalised_polyakov(0.1, 2.3, Nt=4)  # g^2 = 1.74 outside the fit range


def test_free_energy_and_string_tension_fit():
    Nt = 4
    r = np.arange(1, 13, dtype=float)
    a0, a1, sigma = 0.3, 0.25, 0.07
    F_true = a0 - a1 / r + sigma * r
    # C(r) that reproduces F_true after the -T ln 4 shift
    C = np.exp(-Nt * (F_true + np.log(4.0) / Nt))
    F = A.free_energy(C, Nt)
    np.testing.assert_allclose(F, F_true, rtol=0, atol=1e-12)
    (fa0, fa1, fs), cov = A.fit_string_tension(r, F)
    assert (fa0, fa1, fs) == pytest.approx((a0, a1, sigma), abs=1e-10)
    # with noise and errors: within 4 sigma of the truth
    rng = np.random.default_rng(0)
    err = 0.002 * np.ones_like(r)
    (fa0, fa1, fs), cov = A.fit_string_tension(r, F_true + rng.normal(0, 0.002, r.size), err)
    assert abs(fs - sigma) < 4 * np.sqrt(cov[2, 2])
    with pytest.raises(ValueError):
        A.free_energy([0.5, -0.1], Nt)


def test_sigma_ansatz_forms():
    # the paper's first fit: a = 0.6976, b = 0.9990 -> sigma(T_c) ~ a sqrt(1 - b)
    assert A.sigma_ansatz_sqrt(1.0, 0.6976, 0.9990) == pytest.approx(0.6976 * np.sqrt(0.001))
    assert A.sigma_ansatz_sqrt(0.0, 0.6976, 0.9990) == pytest.approx(0.6976)
    assert A.sigma_ansatz_ising(0.0, 1.5541, -0.5122) == 0.0
    assert A.sigma_ansatz_ising(0.25, 1.0, 0.0) == pytest.approx(0.25 ** 0.63)
