"""Pins of the FP64 CPU oracle against facts that do not come from the oracle.

Each test checks one part of the oracle against a library routine, a closed
form, an exact identity or a brute-force case, so that a dropped term, a
wrong sign or index, or a transposed operand in the oracle fails one of them:

* Philox4x32-10       -> cuRAND's host Philox4x32-10 generator (library)
* Haar draws           -> exact laws of the Haar measure on S^3 (marginal CDF,
                          2nd and 4th moments, isotropy) for the hot start,
                          the alpha -> 0 branch and the gauge g(x); <P> = 0
* cold start           -> P = L = C(r) = 1 exactly (definitions, Sec. 2.1/2.2)
* plaquette indices    -> abelian (U(1)-embedded) closed form
* staple               -> sum_x,mu 1/2 Tr(U A) = 24 V P (exact identity)
* gauge invariance     -> P, L, C(r) unchanged by a random g(x) (Sec. 2.2, Eq. 3)
* Polyakov / C(r)      -> constant-link closed form cos(Nt theta); brute force
* Kennedy-Pendleton    -> KS test against the exact density sqrt(1-a0^2)e^{alpha a0},
                          mean I2(alpha)/I1(alpha) (Bessel functions, scipy)
* U_new = X Vhat^+     -> <1/2 Tr(U A)/k> = I2(beta k)/I1(beta k), isotropy
* checkerboard         -> a phase touches only its links; site order irrelevant
* whole chain          -> strong coupling <P> = I2(beta)/I1(beta) at beta = 0.5,
                          weak coupling beta (1 - <P>) -> 3/4
"""
import ctypes
import ctypes.util
import glob
import os

import numpy as np
import pytest
from scipy import integrate, special, stats

from oracle import oracle as O
from paper_1104_5432_gb300 import inputs


# --------------------------------------------------------------------------
# Philox4x32-10 against cuRAND's host generator
# --------------------------------------------------------------------------
def _curand():
    cands = []
    found = ctypes.util.find_library("curand")
    if found:
        cands.append(found)
    for d in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/sbsa-linux/lib",
              "/usr/local/cuda/targets/x86_64-linux/lib"):
        cands += sorted(glob.glob(os.path.join(d, "libcurand.so*")))
    for c in cands:
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand_host_words(lib, seed, offset, n):
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        buf = (ctypes.c_uint32 * n)()
        assert lib.curandGenerate(gen, buf, ctypes.c_size_t(n)) == 0
        return np.array(buf, dtype=np.uint32)
    finally:
        lib.curandDestroyGenerator(gen)


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
@pytest.mark.parametrize("block0", [0, 65536 * 3 + 17, 65536 * (2 ** 32 + 5) + 65533])
def test_philox_matches_curand_host(seed, block0):
    """cuRAND's host Philox generator emits, for output block B (four words),
    Philox4x32-10 of counter (B div 65536 as 64 bits in words 0..1,
    B mod 65536 in word 2, 0) under key (seed lo, seed hi).  The last case
    puts a non-zero value in counter words 0, 1 and 2 at once."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not found")
    nblk = 6
    words = _curand_host_words(lib, seed, 4 * block0, 4 * nblk)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for j in range(nblk):
        B = block0 + j
        hi = B // 65536
        ctr = [hi & 0xFFFFFFFF, hi >> 32, B % 65536, 0]
        np.testing.assert_array_equal(O.philox(ctr, key), words[4 * j:4 * j + 4])


def test_u01_cells():
    # the 2^23 cells are centred: smallest 2^-24, largest 1 - 2^-24, symmetric
    assert O.u01(0) == 2.0 ** -24
    assert O.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    for w in (0x12345678, 0x80000000, 0xDEADBEEF):
        assert O.u01(w) + O.u01(0xFFFFFFFF - w) == 1.0
    # only the top 23 bits matter
    assert O.u01(0x1FF) == O.u01(0)


# --------------------------------------------------------------------------
# start configurations and observables
# --------------------------------------------------------------------------
@pytest.mark.parametrize("Ns,Nt", [(4, 4), (4, 6), (6, 2)])
def test_cold_start_exact(Ns, Nt):
    links = O.init(Ns, Nt, hot=False, seed=0)
    assert O.plaquette(Ns, Nt, links) == 1.0
    m, a, field = O.polyakov(Ns, Nt, links)
    assert m == 1.0 and a == 1.0 and np.all(field == 1.0)
    np.testing.assert_array_equal(O.correlator(Ns, Nt, links, Ns // 2), np.ones(Ns // 2 + 1))


# The Haar measure on SU(2) = S^3 fixes the law of every quaternion the
# oracle draws as "random SU(2)" (hot start, the alpha -> 0 branch of the
# heat bath, the gauge transformation's g(x)).  For a uniform point a on S^3:
#   * each component has the density (2/pi) sqrt(1 - x^2) on [-1, 1], i.e.
#     the CDF 1/2 + (x sqrt(1 - x^2) + arcsin x) / pi;
#   * E[a_i a_j] = delta_ij / 4;
#   * E[a_i^2 a_j^2] = 1/24 (i != j) and E[a_i^4] = 1/8
#     (E[x_1^2 x_2^2] = 1/(n(n+2)), E[x_1^4] = 3/(n(n+2)) on S^(n-1), n = 4);
#   * the direction of the vector part (a1, a2, a3)/|a| is uniform on S^2
#     (cos(theta) and phi uniform) and independent of a0.
# A Box-Muller pair built from cos twice, a second pair drawn from the
# first pair's uniforms, or an angle over half a turn all break one of these.
def _haar_cdf(x):
    x = np.clip(x, -1.0, 1.0)
    return 0.5 + (x * np.sqrt(1.0 - x * x) + np.arcsin(x)) / np.pi


def _check_haar(q):
    """Every law above, at 5 sigma (moments) or p > 1e-4 (KS)."""
    q = np.asarray(q, np.float64).reshape(-1, 4)
    n = q.shape[0]
    np.testing.assert_allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-14)
    for i in range(4):
        assert stats.kstest(q[:, i], _haar_cdf).pvalue > 1e-4, i
    # second moments: diagonal sd sqrt(1/8 - 1/16), off-diagonal sd sqrt(1/24)
    m2 = q.T @ q / n
    sd2 = np.where(np.eye(4) > 0, np.sqrt(1 / 16), np.sqrt(1 / 24)) / np.sqrt(n)
    assert np.all(np.abs(m2 - np.eye(4) / 4) < 5 * sd2), m2
    # fourth moments: E[a_i^4] = 1/8 (sd of a^4: sqrt(105/1920 - 1/64)),
    # E[a_i^2 a_j^2] = 1/24 (sd: sqrt(9/1920 - 1/576))
    q2 = q * q
    m4 = q2.T @ q2 / n
    exp4 = np.where(np.eye(4) > 0, 1 / 8, 1 / 24)
    sd4 = np.where(np.eye(4) > 0, np.sqrt(105 / 1920 - 1 / 64),
                   np.sqrt(9 / 1920 - 1 / 576)) / np.sqrt(n)
    assert np.all(np.abs(m4 - exp4) < 5 * sd4), m4
    # direction of the vector part: uniform on S^2, independent of a0
    v = q[:, 1:]
    u = v / np.linalg.norm(v, axis=1, keepdims=True)
    assert stats.kstest(u[:, 2], stats.uniform(-1, 2).cdf).pvalue > 1e-4
    phi = np.arctan2(u[:, 1], u[:, 0])
    assert stats.kstest(phi, stats.uniform(-np.pi, 2 * np.pi).cdf).pvalue > 1e-4
    for comp in (u, u * u):
        for i in range(3):
            assert abs(np.corrcoef(q[:, 0], comp[:, i])[0, 1]) < 5 / np.sqrt(n)
            assert abs(np.corrcoef(q[:, 0] ** 2, comp[:, i])[0, 1]) < 5 / np.sqrt(n)


def test_haar_pin_detects_broken_draws():
    """The checks above reject the plausible mistakes in a Box-Muller Haar
    draw (guards the pin itself): cos used twice, one pair reused, half-turn
    angles, and three normals instead of four."""
    rng = np.random.default_rng(11)
    n = 100000
    ua, ub, uc, ud = rng.random((4, n))
    r1, r2 = np.sqrt(-2 * np.log(ua)), np.sqrt(-2 * np.log(uc))
    good = np.stack([r1 * np.cos(2 * np.pi * ub), r1 * np.sin(2 * np.pi * ub),
                     r2 * np.cos(2 * np.pi * ud), r2 * np.sin(2 * np.pi * ud)], 1)
    bad = {
        "cos twice": np.stack([r1 * np.cos(2 * np.pi * ub), r1 * np.cos(2 * np.pi * ub),
                               r2 * np.cos(2 * np.pi * ud), r2 * np.cos(2 * np.pi * ud)], 1),
        "pair reused": np.stack([good[:, 0], good[:, 1], good[:, 0], good[:, 1]], 1),
        "half turn": np.stack([r1 * np.cos(np.pi * ub), r1 * np.sin(np.pi * ub),
                               r2 * np.cos(np.pi * ud), r2 * np.sin(np.pi * ud)], 1),
        "three normals": np.stack([good[:, 0], good[:, 1], good[:, 2], np.zeros(n)], 1),
    }
    _check_haar(good / np.linalg.norm(good, axis=1, keepdims=True))
    for name, b in bad.items():
        with pytest.raises(AssertionError):
            _check_haar(b / np.linalg.norm(b, axis=1, keepdims=True))
            pytest.fail(name)


def test_hot_start_is_haar():
    """or_init(hot): every link is a Haar draw (Sec. 2.1 "random SU(2)
    matrix initialization", reading: Haar measure)."""
    Ns = Nt = 12
    links = O.init(Ns, Nt, hot=True, seed=1)
    _check_haar(links)
    # <P> = 0 for independent Haar links (beta = 0), sd of one plaquette 1/2
    P = O.plaquette(Ns, Nt, links)
    assert abs(P) < 5 * 0.5 / np.sqrt(6 * Ns ** 3 * Nt)
    # different seeds give different configurations
    assert not np.array_equal(O.init(4, 4, True, 1), O.init(4, 4, True, 2))


def test_alpha_zero_branch_is_haar():
    """The alpha -> 0 limit of the heat-bath law is the Haar measure: at
    beta = 0 every updated link is a Haar draw (Philox tag 1), whatever the
    staple; and a zero staple at any beta takes the same branch."""
    Ns = Nt = 12
    links = inputs.random_links(Ns, Nt, 5)
    out = []
    for mu in range(4):
        for p in range(2):
            links, trials, cnt = O.heatbath_phase(Ns, Nt, links, 0.0, mu, p, seed=21, sweep=2)
            assert np.all(trials[trials != -2] == 0) and cnt[2] == 0
    _check_haar(links)
    zs = np.array([O.update_from_staple([0, 0, 0, 0], 2.3, seed=8, c0=i, sweep=1)[0]
                   for i in range(40000)])
    _check_haar(zs)


def test_gauge_transform_g_is_haar():
    """or_gauge_transform of a cold start leaves U_0(x) = g(x) g(x+0)^+;
    on even x these are products of disjoint pairs of independent g's, so
    they are independent and Haar exactly when g is."""
    Ns, Nt = 12, 12
    links = O.gauge_transform(Ns, Nt, O.init(Ns, Nt, False, 0), seed=77)
    x = np.arange(Ns ** 3 * Nt) % Ns
    _check_haar(links[x % 2 == 0, 0])


def _abelian(theta):
    """theta[V,4] -> links exp(i theta sigma_3) = (cos theta, 0, 0, sin theta)"""
    q = np.zeros(theta.shape + (4,))
    q[..., 0] = np.cos(theta)
    q[..., 3] = np.sin(theta)
    return np.ascontiguousarray(q)


@pytest.mark.parametrize("Ns,Nt", [(4, 4), (4, 6)])
def test_plaquette_abelian_closed_form(Ns, Nt):
    """For commuting links exp(i theta sigma_3) the plaquette is
    cos(theta_mu(x) + theta_nu(x+mu) - theta_mu(x+nu) - theta_nu(x))."""
    rng = np.random.default_rng(3)
    th = rng.uniform(-np.pi, np.pi, size=(Nt, Ns, Ns, Ns, 4))  # [t,z,y,x,mu]
    links = _abelian(th.reshape(-1, 4))
    axis = {0: 3, 1: 2, 2: 1, 3: 0}  # direction -> array axis of [t,z,y,x]
    tot = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            fwd_mu = lambda a: np.roll(a, -1, axis=axis[mu])
            fwd_nu = lambda a: np.roll(a, -1, axis=axis[nu])
            ang = th[..., mu] + fwd_mu(th[..., nu]) - fwd_nu(th[..., mu]) - th[..., nu]
            tot += np.cos(ang).sum()
    expect = tot / (6 * Ns ** 3 * Nt)
    assert abs(O.plaquette(Ns, Nt, links) - expect) < 1e-14


@pytest.mark.parametrize("Ns,Nt,seed", [(2, 2, 1), (4, 4, 2), (4, 6, 3), (6, 4, 4)])
def test_staple_identity(Ns, Nt, seed):
    """Every plaquette holds four links, so sum_{x,mu} 1/2 Re Tr(U_mu(x) A_mu(x))
    = 4 * 6V * <P> exactly (up to rounding) for ANY configuration."""
    links = inputs.random_links(Ns, Nt, seed)
    V = Ns ** 3 * Nt
    lhs = O.staple_trace_sum(Ns, Nt, links)
    rhs = 24 * V * O.plaquette(Ns, Nt, links)
    assert abs(lhs - rhs) < 1e-12 * V


def test_staple_is_multiple_of_su2():
    links = inputs.random_links(4, 4, 5)
    for lex, mu in [(0, 0), (17, 1), (100, 2), (255, 3)]:
        A = O.staple(4, 4, links, lex, mu)
        assert np.linalg.norm(A) <= 6.0 + 1e-12
    # cold start: each of the six staples is the identity
    cold = O.init(4, 4, False, 0)
    np.testing.assert_array_equal(O.staple(4, 4, cold, 9, 2), [6.0, 0, 0, 0])


@pytest.mark.parametrize("Ns,Nt,sweeps", [(4, 4, 0), (4, 6, 2), (6, 2, 1)])
def test_gauge_invariance(Ns, Nt, sweeps):
    links = O.init(Ns, Nt, True, 11)
    if sweeps:
        links, _, _ = O.heatbath(Ns, Nt, links, 2.2, sweeps, 5)
    g = O.gauge_transform(Ns, Nt, links, 99)
    assert np.max(np.abs(g - links)) > 0.1  # the links really changed
    assert abs(O.plaquette(Ns, Nt, g) - O.plaquette(Ns, Nt, links)) < 1e-14
    m0, a0, f0 = O.polyakov(Ns, Nt, links)
    m1, a1, f1 = O.polyakov(Ns, Nt, g)
    np.testing.assert_allclose(f1, f0, atol=1e-14, rtol=0)
    np.testing.assert_allclose(O.correlator(Ns, Nt, g, Ns // 2),
                               O.correlator(Ns, Nt, links, Ns // 2), atol=1e-14, rtol=0)
    assert np.max(np.abs(np.linalg.norm(g, axis=2) - 1)) < 1e-14


@pytest.mark.parametrize("Nt", [2, 4, 6])
def test_polyakov_constant_links(Nt):
    """U_3(x,t) = W = (cos th, sin th n) for all sites gives L = cos(Nt th)."""
    Ns = 4
    th = 0.37
    n = np.array([0.48, -0.6, 0.64])
    links = O.init(Ns, Nt, False, 0)
    links[:, 3, 0] = np.cos(th)
    links[:, 3, 1:] = np.sin(th) * n
    m, a, field = O.polyakov(Ns, Nt, links)
    np.testing.assert_allclose(field, np.cos(Nt * th), atol=1e-14)
    np.testing.assert_allclose(O.correlator(Ns, Nt, links, 2), np.cos(Nt * th) ** 2, atol=1e-14)


def test_polyakov_single_slice_and_correlator_brute_force():
    """Only U_3(x, t=0) differs from 1, so L(x) = a0(U_3(x,0)); the
    correlator is then checked against a brute-force sum over shifts."""
    Ns, Nt = 6, 4
    links = O.init(Ns, Nt, False, 0)
    q = inputs.random_unit_quaternions(Ns ** 3, 21)
    links[:Ns ** 3, 3, :] = q
    m, a, field = O.polyakov(Ns, Nt, links)
    np.testing.assert_allclose(field, q[:, 0], atol=1e-15)
    assert abs(m - q[:, 0].mean()) < 1e-15 and abs(a - abs(q[:, 0].mean())) < 1e-15
    Lg = q[:, 0].reshape(Ns, Ns, Ns)  # [z,y,x]
    expect = []
    for r in range(Ns // 2 + 1):
        s = 0.0
        for z in range(Ns):
            for y in range(Ns):
                for x in range(Ns):
                    s += Lg[z, y, x] * (Lg[z, y, (x + r) % Ns] + Lg[z, (y + r) % Ns, x]
                                        + Lg[(z + r) % Ns, y, x])
        expect.append(s / (3 * Ns ** 3))
    np.testing.assert_allclose(O.correlator(Ns, Nt, links, Ns // 2), expect, atol=1e-15)
    with pytest.raises(ValueError):
        O.correlator(Ns, Nt, links, Ns // 2 + 1)


# --------------------------------------------------------------------------
# the Kennedy-Pendleton sampler and the link update
# --------------------------------------------------------------------------
def _a0_cdf(alpha):
    """Exact CDF of the density proportional to sqrt(1-a0^2) exp(alpha a0)
    on [-1,1], built with a0 = cos(theta): density sin^2 theta exp(alpha
    (cos theta - 1)) on [0, pi]; normaliser pi I1(alpha) e^-alpha / alpha."""
    z = np.pi * special.ive(1, alpha) / alpha
    th = np.linspace(0.0, np.pi, 4001)
    f = lambda t: np.sin(t) ** 2 * np.exp(alpha * (np.cos(t) - 1.0))
    pieces = [integrate.quad(f, th[i], th[i + 1], epsabs=1e-14)[0] for i in range(len(th) - 1)]
    tail = np.concatenate([[0.0], np.cumsum(pieces)])  # mass in [0, theta]
    assert abs(tail[-1] - z) < 1e-9 * z
    a0_grid = np.cos(th)[::-1]
    cdf_grid = (1.0 - tail / z)[::-1]  # P(a0' <= cos theta) = mass in [theta, pi]

    def cdf(a0):
        return np.interp(a0, a0_grid, cdf_grid)
    return cdf


@pytest.mark.parametrize("alpha", [0.5, 1.0, 5.0, 20.0, 60.0])
def test_kp_sampler_distribution(alpha):
    n = 100000
    a0, trials = O.kp_samples(alpha, seed=1234 + int(alpha * 10), sweep=3, n=n)
    assert np.all(trials >= 1)
    assert np.all((a0 >= -1.0) & (a0 <= 1.0))
    ks = stats.kstest(a0, _a0_cdf(alpha))
    assert ks.pvalue > 1e-4, ks
    mean = special.ive(2, alpha) / special.ive(1, alpha)
    assert abs(a0.mean() - mean) < 5 * a0.std() / np.sqrt(n)


@pytest.mark.parametrize("alpha", [0.01, 0.3, 1.0, 3.0])
def test_creutz_sampler_distribution(alpha):
    """Creutz's draw targets the same density as Kennedy-Pendleton's."""
    n = 100000
    a0, trials = O.kp_samples(alpha, seed=4321 + int(alpha * 100), sweep=2, n=n, creutz=True)
    assert np.all(trials >= 1) and np.all((a0 >= -1.0) & (a0 <= 1.0))
    assert stats.kstest(a0, _a0_cdf(alpha)).pvalue > 1e-4
    mean = special.ive(2, alpha) / special.ive(1, alpha)
    assert abs(a0.mean() - mean) < 5 * a0.std() / np.sqrt(n)
    # acceptance near pi/4 at small alpha, where Kennedy-Pendleton's collapses
    if alpha <= 0.3:
        assert n / trials.sum() > 0.7
        _, kp_trials = O.kp_samples(alpha, seed=1, sweep=2, n=2000)
        assert 2000 / kp_trials.sum() < 0.25


def test_hybrid_strong_coupling_and_tiny_beta():
    """With Creutz's draw below alpha = 1.7 the chain keeps the strong-
    coupling limit, and a vanishing beta no longer hits the trial cap."""
    Ns = Nt = 6
    links = O.init(Ns, Nt, True, 7)
    links, _, _ = O.heatbath(Ns, Nt, links, 0.5, 20, 13, creutz_below=1.7)
    links, p, c = O.heatbath(Ns, Nt, links, 0.5, 400, 13, sweep0=20, creutz_below=1.7)
    b = p.reshape(-1, 20).mean(1)
    u = special.ive(2, 0.5) / special.ive(1, 0.5)
    assert abs(p.mean() - u) < 3 * b.std(ddof=1) / np.sqrt(len(b)) + 2e-4
    assert c[0] / c[1] < 1.5  # ~1.3 trials per update instead of ~2 with KP alone
    new, trials, cnt = O.heatbath_phase(2, 2, O.init(2, 2, True, 4), 1e-9, 1, 0, 3, 0,
                                        creutz_below=1.7)
    assert cnt[2] == 0 and np.all(trials[trials != -2] >= 1)


def test_kp_sampler_rejects_wrong_alpha():
    """The KS test does see a factor-two error in alpha (guards the pin itself)."""
    a0, _ = O.kp_samples(5.0, seed=77, sweep=0, n=100000)
    assert stats.kstest(a0, _a0_cdf(10.0)).pvalue < 1e-10
    assert stats.kstest(a0, _a0_cdf(2.5)).pvalue < 1e-10


def test_update_from_staple_conditional_law():
    """For a fixed staple A = k Vhat, the heat-bath link U satisfies
    1/2 Tr(U Vhat) ~ sqrt(1-a0^2) exp(beta k a0) and the vector part of
    U Vhat is isotropic."""
    beta, k = 2.0, 2.7
    V = inputs.random_unit_quaternions(1, 8)[0]
    A = k * V
    n = 20000
    a0 = np.empty(n)
    vec = np.empty((n, 3))
    # quaternion product written out for the check only: (U Vhat)
    for i in range(n):
        U, t = O.update_from_staple(A, beta, seed=4242, c0=i, sweep=7)
        assert t >= 1
        u0, u1, u2, u3 = U
        v0, v1, v2, v3 = V
        # matrices: U = u0 + i u.sigma; product via 2x2 complex matrices
        Um = np.array([[u0 + 1j * u3, u2 + 1j * u1], [-u2 + 1j * u1, u0 - 1j * u3]])
        Vm = np.array([[v0 + 1j * v3, v2 + 1j * v1], [-v2 + 1j * v1, v0 - 1j * v3]])
        P = Um @ Vm
        a0[i] = 0.5 * (P[0, 0] + P[1, 1]).real
        vec[i] = [0.5 * (P[0, 1] + P[1, 0]).imag, 0.5 * (P[0, 1] - P[1, 0]).real,
                  0.5 * (P[0, 0] - P[1, 1]).imag]
    alpha = beta * k
    expect = special.ive(2, alpha) / special.ive(1, alpha)
    assert abs(a0.mean() - expect) < 5 * a0.std() / np.sqrt(n)
    assert stats.kstest(a0, _a0_cdf(alpha)).pvalue > 1e-4
    np.testing.assert_allclose(a0 ** 2 + (vec ** 2).sum(1), 1.0, atol=1e-13)
    u = vec / np.linalg.norm(vec, axis=1, keepdims=True)
    assert np.all(np.abs(u.mean(0)) < 5 * np.sqrt(1 / 3 / n))
    assert np.all(np.abs((u ** 2).mean(0) - 1 / 3) < 5 * np.sqrt(4 / 45 / n))
    # the direction is independent of a0 (it comes from other random bits)
    for comp in (u, u ** 2):
        for i in range(3):
            assert abs(np.corrcoef(a0, comp[:, i])[0, 1]) < 5 / np.sqrt(n)


def test_update_degenerate_cases():
    # zero staple: Haar draw, zero trials, unit quaternion
    U, t = O.update_from_staple([0, 0, 0, 0], 2.3, seed=1, c0=5, sweep=0)
    assert t == 0 and abs(np.linalg.norm(U) - 1) < 1e-15
    # beta = 0: also the Haar draw (the exact alpha -> 0 limit)
    U2, t2 = O.update_from_staple([1, 0, 0, 0], 0.0, seed=1, c0=5, sweep=0)
    assert t2 == 0 and np.array_equal(U, U2)
    # vanishing alpha > 0: Kennedy-Pendleton rejects every trial -> cap hit
    U3, t3 = O.update_from_staple([1, 0, 0, 0], 1e-9, seed=1, c0=5, sweep=0)
    assert t3 == -1


# --------------------------------------------------------------------------
# phases and sweeps
# --------------------------------------------------------------------------
@pytest.mark.parametrize("mu,parity", [(0, 0), (1, 1), (3, 0), (2, 1)])
def test_phase_touches_only_its_links_and_is_order_free(mu, parity):
    Ns, Nt = 4, 6
    links = inputs.random_links(Ns, Nt, 31)
    new, trials, cnt = O.heatbath_phase(Ns, Nt, links, 2.4, mu, parity, seed=9, sweep=4)
    rev, trials_r, _ = O.heatbath_phase(Ns, Nt, links, 2.4, mu, parity, seed=9, sweep=4,
                                        reverse=True)
    np.testing.assert_array_equal(new, rev)
    np.testing.assert_array_equal(trials, trials_r)
    t, z, y, x = np.meshgrid(range(Nt), range(Ns), range(Ns), range(Ns), indexing="ij")
    par = ((x + y + z + t) % 2).reshape(-1)
    changed = np.any(new != links, axis=2)
    in_phase = np.zeros_like(changed)
    in_phase[par == parity, mu] = True
    np.testing.assert_array_equal(changed, in_phase)
    assert np.all(trials[in_phase] >= 1) and np.all(trials[~in_phase] == -2)
    assert cnt[1] == in_phase.sum() and cnt[0] == trials[in_phase].sum() and cnt[2] == 0
    np.testing.assert_allclose(np.linalg.norm(new, axis=2), 1.0, atol=2e-16 * 8)


def test_sweeps_compose_and_are_deterministic():
    Ns, Nt = 4, 4
    start = O.init(Ns, Nt, True, 3)
    two, p2, c2 = O.heatbath(Ns, Nt, start, 2.3, 2, seed=17, sweep0=0)
    one, p1a, _ = O.heatbath(Ns, Nt, start, 2.3, 1, seed=17, sweep0=0)
    one, p1b, _ = O.heatbath(Ns, Nt, one, 2.3, 1, seed=17, sweep0=1)
    np.testing.assert_array_equal(one, two)
    np.testing.assert_array_equal(np.concatenate([p1a, p1b]), p2)
    again, _, _ = O.heatbath(Ns, Nt, start, 2.3, 2, seed=17, sweep0=0)
    np.testing.assert_array_equal(again, two)
    other, _, _ = O.heatbath(Ns, Nt, start, 2.3, 2, seed=18, sweep0=0)
    assert np.max(np.abs(other - two)) > 0.1
    assert abs(p2[-1] - O.plaquette(Ns, Nt, two)) == 0.0


def test_cap_hit_keeps_links():
    Ns, Nt = 2, 2
    links = inputs.random_links(Ns, Nt, 4)
    new, trials, cnt = O.heatbath_phase(Ns, Nt, links, 1e-9, 1, 0, seed=3, sweep=0)
    np.testing.assert_array_equal(new, links)
    assert cnt[2] == cnt[1] == Ns ** 3 * Nt // 2 and cnt[0] == O.KP_CAP * cnt[1]


def test_zero_staple_takes_haar_branch():
    """Ns = Nt = 2 with U_nu = 1 for nu != 0: the staple of U_0(0) is
    2 * sum_nu U_0(e_nu)^+, which vanishes for three quaternions at 120 deg."""
    Ns, Nt = 2, 2
    links = O.init(Ns, Nt, False, 0)
    s = np.sqrt(3.0) / 2
    for d, q in zip((1, 2, 4), ([1, 0, 0, 0], [-0.5, s, 0, 0], [-0.5, -s, 0, 0])):
        links[d, 0] = q  # lex 1 = (1,0,0,0), 2 = (0,1,0,0), 4 = (0,0,1,0)
    assert np.all(O.staple(Ns, Nt, links, 0, 0) == 0.0)
    new, trials, cnt = O.heatbath_phase(Ns, Nt, links, 2.3, 0, 0, seed=1, sweep=0)
    assert trials[0, 0] == 0
    assert abs(np.linalg.norm(new[0, 0]) - 1) < 1e-15


@pytest.mark.slow
def test_strong_coupling_limit():
    """beta = 0.5: <P> = I2(beta)/I1(beta) up to O(u^5) ~ 1e-4."""
    Ns = Nt = 6
    links = O.init(Ns, Nt, True, 7)
    links, _, _ = O.heatbath(Ns, Nt, links, 0.5, 20, 11)
    links, p, c = O.heatbath(Ns, Nt, links, 0.5, 600, 11, sweep0=20)
    b = p.reshape(-1, 20).mean(1)
    err = b.std(ddof=1) / np.sqrt(len(b))
    u = special.ive(2, 0.5) / special.ive(1, 0.5)
    assert abs(p.mean() - u) < 3 * err + 2e-4, (p.mean(), u, err)
    assert c[2] == 0


@pytest.mark.slow
def test_weak_coupling_limit():
    """beta (1 - <P>) -> 3/4 as beta -> infinity (equipartition over the nine
    physical modes per site); a linear fit in 1/beta over beta = 10, 20, 40
    extrapolates to 3/4 within 0.02."""
    xs, ys, ws = [], [], []
    for beta in (10.0, 20.0, 40.0):
        links = O.init(4, 4, False, 0)
        links, p, _ = O.heatbath(4, 4, links, beta, 300, int(beta))
        p = p[50:]
        b = p.reshape(-1, 25).mean(1)
        xs.append(1 / beta)
        ys.append(beta * (1 - p.mean()))
        ws.append(1 / (beta * b.std(ddof=1) / np.sqrt(len(b))) ** 2)
    A = np.vstack([np.ones(3), xs]).T
    W = np.diag(ws)
    coef = np.linalg.solve(A.T @ W @ A, A.T @ W @ np.array(ys))
    assert abs(coef[0] - 0.75) < 0.02, coef


def test_single_link_entry_matches_phase():
    """The single-link entry point draws what the phase draws."""
    Ns, Nt = 4, 4
    links = inputs.random_links(Ns, Nt, 41)
    new, trials, _ = O.heatbath_phase(Ns, Nt, links, 2.1, 2, 1, seed=6, sweep=3)
    for lex in (1, 2, 77, 254):
        par = sum(int(v) for v in np.unravel_index(lex, (Nt, Ns, Ns, Ns))) % 2
        u, t = O.heatbath_link(Ns, Nt, links, 2.1, 2, lex, seed=6, sweep=3)
        if par == 1:
            np.testing.assert_array_equal(u, new[lex, 2])
            assert t == trials[lex, 2]


def test_single_link_from_hot_start_on_demand():
    """Drawing the staple's links on demand from the hot-start seed gives
    bit for bit what the phase draws on the stored hot start."""
    Ns, Nt = 4, 6
    links = O.init(Ns, Nt, True, 9)
    new, trials, _ = O.heatbath_phase(Ns, Nt, links, 2.5, 0, 0, seed=3, sweep=0)
    par = (np.arange(Ns ** 3 * Nt) % Ns + np.arange(Ns ** 3 * Nt) // Ns % Ns
           + np.arange(Ns ** 3 * Nt) // Ns ** 2 % Ns + np.arange(Ns ** 3 * Nt) // Ns ** 3) % 2
    for lex in np.flatnonzero(par == 0)[::7]:
        u, t = O.heatbath_link_hot(Ns, Nt, 9, 2.5, 0, int(lex), 3, 0)
        np.testing.assert_array_equal(u, new[lex, 0])
        assert t == trials[lex, 0]
    # other directions agree with the single-link entry on the stored links
    for mu, lex in ((3, 5), (1, 77), (2, 140)):
        u, t = O.heatbath_link_hot(Ns, Nt, 9, 1.7, mu, lex, 4, 2)
        v, tv = O.heatbath_link(Ns, Nt, links, 1.7, mu, lex, 4, 2)
        np.testing.assert_array_equal(u, v)
        assert t == tv
