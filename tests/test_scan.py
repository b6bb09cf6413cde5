"""Host post-processing of the finite-temperature scan (Sec. 2.2): binned
jackknife, the critical coupling, two-loop scale setting and the string
tension fit, against closed forms and synthetic data of known parameters."""
import math

import numpy as np
import pytest

from paper_1104_5432_gb300 import analysis, scan


def test_jackknife_of_independent_bins():
    rng = np.random.default_rng(3)
    x = rng.normal(1.5, 0.2, size=(400, 3))
    m, e, s = scan.jackknife(x)
    assert s.shape == (400, 3)
    np.testing.assert_allclose(m, x.mean(0))
    # for the mean the jackknife error is the standard error exactly
    np.testing.assert_allclose(e, x.std(0, ddof=1) / np.sqrt(400), rtol=1e-12)
    # a nonlinear function: error propagation to first order
    m2, e2, _ = scan.jackknife(x[:, 0], np.log)
    assert e2 == pytest.approx(e[0] / m[0], rel=0.05)


def test_two_loop_scale_setting():
    """d ln(a Lambda)/d beta = b1 / (2 b0^2 beta) - 1 / (8 b0) for g^2 = 4/beta,
    with the SU(2) coefficients b0 = 22/(48 pi^2), b1 = (34/3) 4/(16 pi^2)^2."""
    assert scan.B0 == pytest.approx(22 / (48 * math.pi ** 2))
    assert scan.B1 == pytest.approx(34 / 3 * 4 / (16 * math.pi ** 2) ** 2)
    for b in (2.2, 2.5, 3.0):
        h = 1e-5
        d = (np.log(scan.lattice_spacing(b + h)) - np.log(scan.lattice_spacing(b - h))) / (2 * h)
        assert d == pytest.approx(scan.B1 / (2 * scan.B0 ** 2 * b) - 1 / (8 * scan.B0), rel=1e-6)
    assert scan.t_over_tc(2.3, 2.3) == pytest.approx(1.0)
    assert scan.t_over_tc(2.4, 2.3) > 1.0 > scan.t_over_tc(2.2, 2.3)


def test_beta_critical_at_half_the_largest_value():
    """A symmetric rise (tanh) crosses half its height at its centre, also
    when single couplings past it fall back (domain walls)."""
    betas = np.round(np.arange(2.20, 2.405, 0.01), 2)
    for bc in (2.2873, 2.30, 2.3456):
        y = 0.1 * (1 + np.tanh((betas - bc) / 0.015))
        assert scan.beta_critical(betas, y) == pytest.approx(bc, abs=0.003)
        dips = y.copy()
        dips[-1] = dips[-4] = 0.03
        assert scan.beta_critical(betas, dips) == pytest.approx(bc, abs=0.003)
    assert scan.beta_critical([2.2, 2.3], [0.5, 0.1]) == 2.2


def test_string_tension_fit_recovers_known_parameters():
    """Bins of C(r) = exp(-F(r)/T) / 4 with F = a0 - a1/r + sigma r and
    multiplicative noise: the fit returns sigma within 3 jackknife errors and
    stops where the correlator drowns in noise."""
    rng = np.random.default_rng(7)
    Nt = 4
    T = 1 / Nt
    a0, a1, sigma = 0.6, 0.25, 0.15
    r = np.arange(0, 25)
    F = a0 - a1 / np.maximum(r, 1) + sigma * r
    C = np.exp(-F / T) / 4
    nb = 40
    noise = 1e-5  # absolute, as from a finite number of sweeps
    bins = C[None, :] * (1 + 0.01 * rng.standard_normal((nb, len(r)))) \
        + noise * rng.standard_normal((nb, len(r)))
    fit = scan.fit_sigma(bins, Nt, rmin=2)
    assert fit is not None
    assert abs(fit["sigma"] - sigma) < 3 * fit["sigma_err"] + 1e-3, fit
    assert fit["sigma_err"] < 0.01
    lo, hi = fit["r_range"]
    assert lo == 2 and 8 <= hi <= 16  # beyond hi the noise exceeds 30% of C(r)
    # a flat F (deconfined) leaves sigma compatible with zero
    flat = np.full((nb, len(r)), 0.3) * (1 + 0.002 * rng.standard_normal((nb, len(r))))
    fit0 = scan.fit_sigma(flat, Nt)
    assert abs(fit0["sigma"]) < 3 * fit0["sigma_err"] + 1e-4


def test_analyse_and_table():
    rng = np.random.default_rng(1)
    betas = [2.2, 2.25, 2.3, 2.35, 2.4]
    nb, n, rmax, Nt = 20, len(betas), 8, 4
    La = np.array([0.01, 0.02, 0.06, 0.12, 0.16])
    r = np.arange(rmax + 1)
    C = np.stack([np.exp(-(0.4 + 0.1 * (0.4 - k * 0.1) * r) * Nt) for k in range(n)])
    res = {"betas": betas, "Nt": Nt,
           "plaquette": 0.6 + 0.001 * rng.standard_normal((nb, n)),
           "L": 0.001 * rng.standard_normal((nb, n)),
           "L_abs": La + 0.001 * rng.standard_normal((nb, n)),
           "C": C[None] * (1 + 0.01 * rng.standard_normal((nb, n, rmax + 1)))}
    an = scan.analyse(res)
    assert 2.25 < an["beta_c"] < 2.35
    assert [row["beta"] for row in an["rows"]] == betas
    t = scan.table(an)
    assert t.count("\n") == n + 1 and "sigma" in t
