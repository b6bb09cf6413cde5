/*
 * su2_oracle.c -- plain, slow, FP64 CPU oracle for the SU(2) pure-gauge
 * heat-bath method of Cardoso, Cardoso & Bicudo, "Finite temperature lattice
 * QCD with GPUs" (Excited QCD 2011): random SU(2) start, heat-bath sweeps,
 * mean plaquette per sweep (Sec. 2.1), Polyakov loop (Sec. 2.2, Eq. 1) and
 * the Polyakov-loop correlator behind the colour-averaged free energy
 * (Sec. 2.2, Eq. 3).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may include, link,
 * load or call this file.  Only the test-suite, the package's smoke check and
 * the benchmark's CPU-baseline leg use it.  It shares no code, header, table
 * or constant generator with the CUDA implementation.
 *
 * Every function here is pinned by tests/test_oracle_pins.py to something
 * other than itself (closed forms, cuRAND's Philox, exact distributions,
 * brute force on tiny lattices, invariances); none is "parity unpinned".
 *
 * Everything is written the obvious way: links are kept as quaternions in
 * the canonical host layout but every group operation is done on explicit
 * 2x2 complex matrices, sites are visited in lexicographic order, sums use
 * Neumaier compensation.  No blocking, fusion or reordering.
 *
 * The paper defers the algorithmic details to its companion paper, so the
 * following readings are fixed here (they are listed with their reasons in
 * the design notes of the repository):
 *   action     S = beta * sum_P (1 - 1/2 Re Tr U_P),  beta = 4/g^2
 *   link       quaternion a -> U = [[a0 + i a3, a2 + i a1], [-a2 + i a1, a0 - i a3]]
 *   lattice    extents (Ns,Ns,Ns,Nt) for (x,y,z,t); lex = x+Ns(y+Ns(z+Ns t));
 *              parity = (x+y+z+t) mod 2
 *   layout     host links double[V][4][4]: ((lex*4+mu)*4 + component)
 *   sweep      phases (mu,parity) = (0,0),(0,1),(1,0),(1,1),...,(3,1)
 *   heat bath  Kennedy-Pendleton draw of a0 from sqrt(1-a0^2) exp(alpha a0)
 *              (optionally Creutz's draw below a chosen alpha),
 *              alpha = beta*k, k = sqrt(det A) for the staple sum A;
 *              new link U = X Vhat^dagger, Vhat = A/k, then normalised
 *   RNG        Philox4x32-10, key = (seed lo, seed hi), counter =
 *              (lex*4+mu, sweep lo, tag<<24 | trial, sweep hi);
 *              tag 0 = KP trial, 1 = Haar draw when alpha is negligible,
 *              2 = hot start, 3 = random gauge transformation;
 *              uniform(w) = ((w >> 9) + 0.5) * 2^-23 from the top 23 bits;
 *              the direction of the new link uses the 9 low bits of the
 *              four words of the trial-0 block: u1 from words 0,1 and u2
 *              from words 2,3, each ((hi9 << 9 | lo9) + 0.5) * 2^-18
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_KP_CAP 4096
#define OR_ALPHA_HAAR 1e-12

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its definition:
 * ten rounds of two 32x32->64 multiplications whose high halves are mixed
 * with the other two counter words and the round key; the key is bumped by
 * the Weyl constants between rounds.                                      */
/* ------------------------------------------------------------------ */
void or_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform in (0,1): the top 23 bits of a word, centred in their cell */
double or_u01(uint32_t w)
{
    return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0);
}

static void draw_words(uint64_t seed, uint32_t c0, uint64_t sweep, uint32_t tag,
                       uint32_t trial, uint32_t w[4])
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t ctr[4] = { c0, (uint32_t)sweep, (tag << 24) | trial, (uint32_t)(sweep >> 32) };
    or_philox(ctr, key, w);
}

static void draw(uint64_t seed, uint32_t c0, uint64_t sweep, uint32_t tag,
                 uint32_t trial, double u[4])
{
    uint32_t w[4];
    draw_words(seed, c0, sweep, tag, trial, w);
    for (int i = 0; i < 4; ++i) u[i] = or_u01(w[i]);
}

/* the two direction uniforms from the low 9 bits of a block's words */
static void spare_uniforms(const uint32_t w[4], double *u1, double *u2)
{
    uint32_t k1 = ((w[0] & 511u) << 9) | (w[1] & 511u);
    uint32_t k2 = ((w[2] & 511u) << 9) | (w[3] & 511u);
    *u1 = ((double)k1 + 0.5) / 262144.0;
    *u2 = ((double)k2 + 0.5) / 262144.0;
}

/* Box-Muller: two uniforms -> two independent standard normals */
static void box_muller(double ua, double ub, double *na, double *nb)
{
    double r = sqrt(-2.0 * log(ua));
    *na = r * cos(2.0 * M_PI * ub);
    *nb = r * sin(2.0 * M_PI * ub);
}

/* ------------------------------------------------------------------ */
/* 2x2 complex matrices                                                */
/* ------------------------------------------------------------------ */
typedef struct { double complex e[2][2]; } mat2;

static mat2 m_from_quat(const double a[4])
{
    mat2 m;
    m.e[0][0] = a[0] + I * a[3];
    m.e[0][1] = a[2] + I * a[1];
    m.e[1][0] = -a[2] + I * a[1];
    m.e[1][1] = a[0] - I * a[3];
    return m;
}

/* projection of any 2x2 matrix onto the real span of {1, i sigma_k} */
static void m_to_quat(const mat2 *m, double a[4])
{
    a[0] = 0.5 * creal(m->e[0][0] + m->e[1][1]);
    a[1] = 0.5 * cimag(m->e[0][1] + m->e[1][0]);
    a[2] = 0.5 * creal(m->e[0][1] - m->e[1][0]);
    a[3] = 0.5 * cimag(m->e[0][0] - m->e[1][1]);
}

static mat2 m_mul(const mat2 *a, const mat2 *b)
{
    mat2 c;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            c.e[i][j] = a->e[i][0] * b->e[0][j] + a->e[i][1] * b->e[1][j];
    return c;
}

static mat2 m_dag(const mat2 *a)
{
    mat2 c;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            c.e[i][j] = conj(a->e[j][i]);
    return c;
}

static mat2 m_add(const mat2 *a, const mat2 *b)
{
    mat2 c;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            c.e[i][j] = a->e[i][j] + b->e[i][j];
    return c;
}

static mat2 m_scale(const mat2 *a, double s)
{
    mat2 c;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            c.e[i][j] = a->e[i][j] * s;
    return c;
}

static mat2 m_zero(void)
{
    mat2 c;
    memset(&c, 0, sizeof c);
    return c;
}

static mat2 m_one(void)
{
    mat2 c = m_zero();
    c.e[0][0] = 1.0;
    c.e[1][1] = 1.0;
    return c;
}

static double m_half_retr(const mat2 *a)
{
    return 0.5 * creal(a->e[0][0] + a->e[1][1]);
}

/* ------------------------------------------------------------------ */
/* lattice geometry                                                   */
/* ------------------------------------------------------------------ */
typedef struct { int L[4]; long V; } geom;

static geom mkgeom(int Ns, int Nt)
{
    geom g;
    g.L[0] = g.L[1] = g.L[2] = Ns;
    g.L[3] = Nt;
    g.V = (long)Ns * Ns * Ns * Nt;
    return g;
}

static long lex_of(const geom *g, const int c[4])
{
    return c[0] + (long)g->L[0] * (c[1] + (long)g->L[1] * (c[2] + (long)g->L[2] * c[3]));
}

static void coords_of(const geom *g, long lex, int c[4])
{
    for (int d = 0; d < 4; ++d) {
        c[d] = (int)(lex % g->L[d]);
        lex /= g->L[d];
    }
}

/* lex index of x + s*e_d, periodic */
static long shifted(const geom *g, const int c[4], int d, int s)
{
    int n[4] = { c[0], c[1], c[2], c[3] };
    n[d] = ((n[d] + s) % g->L[d] + g->L[d]) % g->L[d];
    return lex_of(g, n);
}

static long shifted2(const geom *g, const int c[4], int d1, int s1, int d2, int s2)
{
    int n[4] = { c[0], c[1], c[2], c[3] };
    n[d1] = ((n[d1] + s1) % g->L[d1] + g->L[d1]) % g->L[d1];
    n[d2] = ((n[d2] + s2) % g->L[d2] + g->L[d2]) % g->L[d2];
    return lex_of(g, n);
}

static mat2 link(const double *links, long lex, int mu)
{
    return m_from_quat(links + (lex * 4 + mu) * 4);
}

static void store_link(double *links, long lex, int mu, const double a[4])
{
    memcpy(links + (lex * 4 + mu) * 4, a, 4 * sizeof(double));
}

/* Neumaier-compensated running sum */
typedef struct { double s, c; } nsum;
static void nadd(nsum *acc, double v)
{
    double t = acc->s + v;
    if (fabs(acc->s) >= fabs(v)) acc->c += (acc->s - t) + v;
    else acc->c += (v - t) + acc->s;
    acc->s = t;
}
static double nval(const nsum *acc) { return acc->s + acc->c; }

/* ------------------------------------------------------------------ */
/* start configurations                                               */
/* ------------------------------------------------------------------ */

/* Haar-random SU(2) element from four normals of one Philox block */
static void haar_quat(const double u[4], double a[4])
{
    double n[4];
    box_muller(u[0], u[1], &n[0], &n[1]);
    box_muller(u[2], u[3], &n[2], &n[3]);
    double r = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2] + n[3] * n[3]);
    for (int i = 0; i < 4; ++i) a[i] = n[i] / r;
}

/* start = 0: cold (every link the identity); start = 1: hot (Haar links,
 * "random SU(2) matrix initialization", Sec. 2.1), Philox tag 2. */
int or_init(int Ns, int Nt, int start, uint64_t seed, double *links)
{
    geom g = mkgeom(Ns, Nt);
    for (long lex = 0; lex < g.V; ++lex)
        for (int mu = 0; mu < 4; ++mu) {
            double a[4] = { 1.0, 0.0, 0.0, 0.0 };
            if (start == 1) {
                double u[4];
                draw(seed, (uint32_t)(lex * 4 + mu), 0, 2, 0, u);
                haar_quat(u, a);
            }
            store_link(links, lex, mu, a);
        }
    return 0;
}

/* U_mu(x) -> g(x) U_mu(x) g(x+mu)^dagger with Haar g(x) (Philox tag 3) */
void or_gauge_transform(int Ns, int Nt, double *links, uint64_t seed)
{
    geom g = mkgeom(Ns, Nt);
    mat2 *gm = malloc(sizeof(mat2) * g.V);
    for (long lex = 0; lex < g.V; ++lex) {
        double u[4], a[4];
        draw(seed, (uint32_t)(lex * 4), 0, 3, 0, u);
        haar_quat(u, a);
        gm[lex] = m_from_quat(a);
    }
    double *out = malloc(sizeof(double) * g.V * 16);
    for (long lex = 0; lex < g.V; ++lex) {
        int c[4];
        coords_of(&g, lex, c);
        for (int mu = 0; mu < 4; ++mu) {
            mat2 U = link(links, lex, mu);
            mat2 gd = m_dag(&gm[shifted(&g, c, mu, 1)]);
            mat2 t = m_mul(&gm[lex], &U);
            mat2 r = m_mul(&t, &gd);
            double a[4];
            m_to_quat(&r, a);
            memcpy(out + (lex * 4 + mu) * 4, a, sizeof a);
        }
    }
    memcpy(links, out, sizeof(double) * g.V * 16);
    free(out);
    free(gm);
}

/* ------------------------------------------------------------------ */
/* staple and the heat-bath draw                                      */
/* ------------------------------------------------------------------ */

/* Where the staple reads its links: an array in the canonical layout, or
 * (links == NULL) the hot start of or_init with key hot_seed, drawn link
 * by link on demand. */
typedef struct { const double *links; uint64_t hot_seed; } linksrc;

static mat2 src_link(const linksrc *src, long lex, int mu)
{
    if (src->links) return link(src->links, lex, mu);
    double u[4], a[4];
    draw(src->hot_seed, (uint32_t)(lex * 4 + mu), 0, 2, 0, u);
    haar_quat(u, a);
    return m_from_quat(a);
}

/* A_mu(x) = sum_{nu != mu} [ U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
 *                          + U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu) ]
 * so that Re Tr(U_mu(x) A_mu(x)) collects every plaquette holding U_mu(x). */
static mat2 staple_from(const geom *g, const linksrc *src, const int c[4], int mu)
{
    mat2 A = m_zero();
    long x = lex_of(g, c);
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        mat2 a = src_link(src, shifted(g, c, mu, 1), nu);
        mat2 b = src_link(src, shifted(g, c, nu, 1), mu);
        mat2 cc = src_link(src, x, nu);
        mat2 bd = m_dag(&b), cd = m_dag(&cc);
        mat2 t = m_mul(&a, &bd);
        mat2 up = m_mul(&t, &cd);

        mat2 d = src_link(src, shifted2(g, c, mu, 1, nu, -1), nu);
        mat2 e = src_link(src, shifted(g, c, nu, -1), mu);
        mat2 f = src_link(src, shifted(g, c, nu, -1), nu);
        mat2 dd = m_dag(&d), ed = m_dag(&e);
        mat2 s = m_mul(&dd, &ed);
        mat2 lo = m_mul(&s, &f);

        A = m_add(&A, &up);
        A = m_add(&A, &lo);
    }
    return A;
}

static mat2 staple(const geom *g, const double *links, const int c[4], int mu)
{
    linksrc src = { links, 0 };
    return staple_from(g, &src, c, mu);
}

/* Kennedy-Pendleton draw of delta = 1 - a0 with density proportional to
 * sqrt(delta (2-delta)) exp(-alpha delta) on [0,2]  (heat-bath step of
 * Sec. 2.1; Kennedy & Pendleton, Phys. Lett. B156 (1985) 393).
 * Trial t uses Philox tag 0 with trial field t: lambda^2 = -(ln r1 +
 * cos^2(2 pi r2) ln r3) / (2 alpha), accepted when r4^2 <= 1 - lambda^2,
 * then delta = 2 lambda^2.  Returns the number of trials used, or -1 when
 * OR_KP_CAP trials were all rejected. */
static int kp_delta(double alpha, uint64_t seed, uint32_t c0, uint64_t sweep, double *delta)
{
    for (int t = 0; t < OR_KP_CAP; ++t) {
        double r[4];
        draw(seed, c0, sweep, 0, (uint32_t)t, r);
        double cs = cos(2.0 * M_PI * r[1]);
        double lambda2 = -(log(r[0]) + cs * cs * log(r[2])) / (2.0 * alpha);
        if (r[3] * r[3] <= 1.0 - lambda2) {
            *delta = 2.0 * lambda2;
            return t + 1;
        }
    }
    return -1;
}

/* Creutz's draw (Phys. Rev. D21 (1980) 2308) of delta = 1 - a0 for the same
 * density: a0 from exp(alpha a0) on [-1,1] by inversion, x = 1 - r1 (1 -
 * exp(-2 alpha)), a0 = 1 + ln(x)/alpha, accepted when r4^2 <= 1 - a0^2 =
 * delta (2 - delta).  Trial t uses the same Philox block as a
 * Kennedy-Pendleton trial t (tag 0): r1 = word 0, r4 = word 3.
 * Returns the number of trials used, or -1 after OR_KP_CAP rejections. */
static int creutz_delta(double alpha, uint64_t seed, uint32_t c0, uint64_t sweep, double *delta)
{
    double q = -expm1(-2.0 * alpha);
    for (int t = 0; t < OR_KP_CAP; ++t) {
        double r[4];
        draw(seed, c0, sweep, 0, (uint32_t)t, r);
        double d = -log1p(-r[0] * q) / alpha;
        if (r[3] * r[3] <= d * (2.0 - d)) {
            *delta = d;
            return t + 1;
        }
    }
    return -1;
}

/* New link from the staple sum A (as a matrix).  Returns trials (>= 1),
 * 0 for the Haar draw (alpha below OR_ALPHA_HAAR), or -1 on a cap hit, in
 * which case *unew is left untouched. */
/* creutz_below: alpha below which Creutz's draw replaces Kennedy-Pendleton's
 * (0 = Kennedy-Pendleton everywhere) */
static int update_from_staple(const mat2 *A, double beta, uint64_t seed, uint32_t c0,
                              uint64_t sweep, double creutz_below, double unew[4])
{
    double k = sqrt(creal(A->e[0][0] * A->e[1][1] - A->e[0][1] * A->e[1][0]));
    double alpha = beta * k;
    double u[4];
    if (!(alpha >= OR_ALPHA_HAAR)) {
        draw(seed, c0, sweep, 1, 0, u);
        haar_quat(u, unew);
        return 0;
    }
    double delta;
    int trials = alpha < creutz_below ? creutz_delta(alpha, seed, c0, sweep, &delta)
                                      : kp_delta(alpha, seed, c0, sweep, &delta);
    if (trials < 0) return -1;

    uint32_t w0[4];
    double u1, u2;
    draw_words(seed, c0, sweep, 0, 0, w0);
    spare_uniforms(w0, &u1, &u2);
    double cth = 2.0 * u1 - 1.0;
    double sth = sqrt((1.0 - cth) * (1.0 + cth));
    double phi = 2.0 * M_PI * u2;
    double vlen = sqrt(delta * (2.0 - delta));
    double xq[4] = { 1.0 - delta, vlen * sth * cos(phi), vlen * sth * sin(phi), vlen * cth };

    mat2 X = m_from_quat(xq);
    mat2 Vh = m_scale(A, 1.0 / k);
    mat2 Vd = m_dag(&Vh);
    mat2 Un = m_mul(&X, &Vd);
    double a[4];
    m_to_quat(&Un, a);
    double n = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3]);
    for (int i = 0; i < 4; ++i) unew[i] = a[i] / n;
    return trials;
}

/* One phase: every U_mu(x) with parity(x) == parity gets a heat-bath
 * update from the current configuration.  Links of one phase share no
 * staple, so the visiting order does not matter; reverse != 0 walks the
 * sites backwards (used only to check that claim).
 * trials_out (nullable, [V*4] indexed lex*4+mu): trials used, 0 for a Haar
 * draw, -1 for a cap hit; untouched for links outside the phase.
 * counters (nullable): [0] += trials, [1] += links visited, [2] += cap hits. */
int or_heatbath_phase(int Ns, int Nt, double *links, double beta, int mu, int parity,
                      uint64_t seed, uint64_t sweep, int reverse, double creutz_below,
                      int32_t *trials_out, uint64_t *counters)
{
    geom g = mkgeom(Ns, Nt);
    for (long i = 0; i < g.V; ++i) {
        long lex = reverse ? g.V - 1 - i : i;
        int c[4];
        coords_of(&g, lex, c);
        if (((c[0] + c[1] + c[2] + c[3]) & 1) != parity) continue;
        mat2 A = staple(&g, links, c, mu);
        double unew[4];
        uint32_t c0 = (uint32_t)(lex * 4 + mu);
        int tr = update_from_staple(&A, beta, seed, c0, sweep, creutz_below, unew);
        if (tr >= 0) store_link(links, lex, mu, unew);
        if (trials_out) trials_out[lex * 4 + mu] = tr;
        if (counters) {
            counters[0] += (uint64_t)(tr > 0 ? tr : (tr < 0 ? OR_KP_CAP : 0));
            counters[1] += 1;
            counters[2] += (tr < 0);
        }
    }
    return 0;
}

/* The link the phase (mu, parity(x)) would draw for U_mu(x) alone, from
 * the configuration as given (for sampled checks on large lattices).
 * Returns trials as or_update_from_staple; unew is untouched on a cap hit. */
int or_heatbath_link(int Ns, int Nt, const double *links, double beta, int mu, long lex,
                     uint64_t seed, uint64_t sweep, double creutz_below, double unew[4])
{
    geom g = mkgeom(Ns, Nt);
    int c[4];
    coords_of(&g, lex, c);
    mat2 A = staple(&g, links, c, mu);
    return update_from_staple(&A, beta, seed, (uint32_t)(lex * 4 + mu), sweep, creutz_below, unew);
}

/* The link the first phase after a hot start, (mu, parity) = (0, 0) at
 * sweep 0 when lex is an even site, draws for U_mu(lex): the same as
 * or_heatbath_link on or_init(Ns, Nt, 1, init_seed), but only the 18 links
 * of the staple are drawn, so lattices too large to hold on the host
 * (128^4: 34 GB of links) can be checked at sampled sites. */
int or_heatbath_link_hot(int Ns, int Nt, uint64_t init_seed, double beta, int mu, long lex,
                         uint64_t seed, uint64_t sweep, double creutz_below, double unew[4])
{
    geom g = mkgeom(Ns, Nt);
    int c[4];
    coords_of(&g, lex, c);
    linksrc src = { NULL, init_seed };
    mat2 A = staple_from(&g, &src, c, mu);
    return update_from_staple(&A, beta, seed, (uint32_t)(lex * 4 + mu), sweep, creutz_below, unew);
}

/* Test hook for the sampler: the link drawn by the heat-bath step for a
 * given staple quaternion A (any real multiple of an SU(2) element). */
int or_update_from_staple(const double A[4], double beta, uint64_t seed, uint32_t c0,
                          uint64_t sweep, double creutz_below, double unew[4])
{
    mat2 Am = m_from_quat(A);
    return update_from_staple(&Am, beta, seed, c0, sweep, creutz_below, unew);
}

/* Test hook: n KP draws of a0 = 1 - delta for a fixed alpha, drawn with
 * counter words c0 = i (i = 0..n-1) and the given sweep. */
void or_kp_samples(double alpha, uint64_t seed, uint64_t sweep, long n, int creutz, double *a0,
                   int32_t *trials)
{
    for (long i = 0; i < n; ++i) {
        double delta = NAN;
        int t = creutz ? creutz_delta(alpha, seed, (uint32_t)i, sweep, &delta)
                       : kp_delta(alpha, seed, (uint32_t)i, sweep, &delta);
        a0[i] = 1.0 - delta;
        if (trials) trials[i] = t;
    }
}

/* ------------------------------------------------------------------ */
/* observables                                                        */
/* ------------------------------------------------------------------ */

/* mean plaquette (1/6V) sum_x sum_{mu<nu} 1/2 Re Tr U_mu(x) U_nu(x+mu)
 * U_mu(x+nu)^+ U_nu(x)^+  ("mean average plaquette", Sec. 2.1) */
double or_plaquette(int Ns, int Nt, const double *links)
{
    geom g = mkgeom(Ns, Nt);
    nsum acc = { 0.0, 0.0 };
    for (long lex = 0; lex < g.V; ++lex) {
        int c[4];
        coords_of(&g, lex, c);
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu) {
                mat2 a = link(links, lex, mu);
                mat2 b = link(links, shifted(&g, c, mu, 1), nu);
                mat2 cc = link(links, shifted(&g, c, nu, 1), mu);
                mat2 d = link(links, lex, nu);
                mat2 cd = m_dag(&cc), dd = m_dag(&d);
                mat2 t1 = m_mul(&a, &b);
                mat2 t2 = m_mul(&t1, &cd);
                mat2 p = m_mul(&t2, &dd);
                nadd(&acc, m_half_retr(&p));
            }
    }
    return nval(&acc) / (6.0 * (double)g.V);
}

/* sum over x and mu of 1/2 Re Tr(U_mu(x) A_mu(x)); every plaquette holds
 * four links, so this equals 4 * 6V * plaquette for any configuration. */
double or_staple_trace_sum(int Ns, int Nt, const double *links)
{
    geom g = mkgeom(Ns, Nt);
    nsum acc = { 0.0, 0.0 };
    for (long lex = 0; lex < g.V; ++lex) {
        int c[4];
        coords_of(&g, lex, c);
        for (int mu = 0; mu < 4; ++mu) {
            mat2 A = staple(&g, links, c, mu);
            mat2 U = link(links, lex, mu);
            mat2 p = m_mul(&U, &A);
            nadd(&acc, m_half_retr(&p));
        }
    }
    return nval(&acc);
}

/* staple quaternion of one link (the projection of A, exact since A is a
 * real multiple of an SU(2) element) */
void or_staple(int Ns, int Nt, const double *links, long lex, int mu, double out[4])
{
    geom g = mkgeom(Ns, Nt);
    int c[4];
    coords_of(&g, lex, c);
    mat2 A = staple(&g, links, c, mu);
    m_to_quat(&A, out);
}

/* Polyakov loop L(x) = 1/2 Re Tr prod_{t=0}^{Nt-1} U_3(x,t) for every
 * spatial site (Sec. 2.2, Eq. 1; product ordered t = 0 .. Nt-1).
 * Lfield (nullable) gets the Ns^3 values in lexicographic (x,y,z) order.
 * Returns the volume mean; *abs_mean (nullable) gets its modulus. */
double or_polyakov(int Ns, int Nt, const double *links, double *abs_mean, double *Lfield)
{
    geom g = mkgeom(Ns, Nt);
    long Vs = (long)Ns * Ns * Ns;
    nsum acc = { 0.0, 0.0 };
    for (long s = 0; s < Vs; ++s) {
        mat2 P = m_one();
        for (int t = 0; t < Nt; ++t) {
            mat2 U = link(links, s + Vs * t, 3);
            P = m_mul(&P, &U);
        }
        double L = m_half_retr(&P);
        if (Lfield) Lfield[s] = L;
        nadd(&acc, L);
    }
    double m = nval(&acc) / (double)Vs;
    if (abs_mean) *abs_mean = fabs(m);
    (void)g;
    return m;
}

/* C(r) = (1/(3 Ns^3)) sum_x sum_{i=x,y,z} L(x) L(x + r e_i), r = 0..rmax,
 * periodic; for SU(2) the traces are real, so 1/4 Tr L(y) Tr L^+(x) of
 * Sec. 2.2, Eq. 3 is the product of the two normalised loops. */
int or_correlator(int Ns, int Nt, const double *links, int rmax, double *out)
{
    if (rmax < 0 || rmax > Ns / 2) return -1;
    long Vs = (long)Ns * Ns * Ns;
    double *L = malloc(sizeof(double) * Vs);
    or_polyakov(Ns, Nt, links, NULL, L);
    for (int r = 0; r <= rmax; ++r) {
        nsum acc = { 0.0, 0.0 };
        for (long s = 0; s < Vs; ++s) {
            int x = (int)(s % Ns), y = (int)((s / Ns) % Ns), z = (int)(s / ((long)Ns * Ns));
            long sx = ((x + r) % Ns) + (long)Ns * (y + (long)Ns * z);
            long sy = x + (long)Ns * (((y + r) % Ns) + (long)Ns * z);
            long sz = x + (long)Ns * (y + (long)Ns * ((z + r) % Ns));
            nadd(&acc, L[s] * L[sx]);
            nadd(&acc, L[s] * L[sy]);
            nadd(&acc, L[s] * L[sz]);
        }
        out[r] = nval(&acc) / (3.0 * (double)Vs);
    }
    free(L);
    return 0;
}

/* nsweeps full sweeps with sweep indices sweep0 .. sweep0+nsweeps-1; the
 * mean plaquette after each sweep goes to plaq_out (nullable). */
int or_heatbath(int Ns, int Nt, double *links, double beta, int nsweeps, uint64_t seed,
                uint64_t sweep0, double creutz_below, double *plaq_out, uint64_t *counters)
{
    for (int s = 0; s < nsweeps; ++s) {
        for (int mu = 0; mu < 4; ++mu)
            for (int p = 0; p < 2; ++p)
                or_heatbath_phase(Ns, Nt, links, beta, mu, p, seed, sweep0 + (uint64_t)s, 0,
                                  creutz_below, NULL, counters);
        if (plaq_out) plaq_out[s] = or_plaquette(Ns, Nt, links);
    }
    return 0;
}
