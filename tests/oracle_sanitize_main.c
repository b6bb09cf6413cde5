/*
 * Driver for the sanitizer test of the CPU oracle: compiled together with
 * oracle/su2_oracle.c under -fsanitize=address,undefined, it calls every
 * exported oracle function on small and ragged lattices (2^4, 4^3 x 6,
 * 6^3 x 2) in both samplers, at the edge cases (beta = 0, beta = 1e-9 with
 * the trial cap, rmax = Ns/2), and exits 0 only if the results are finite
 * and the links stay unit quaternions.  Any out-of-bounds access or
 * undefined behaviour aborts the run.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

void or_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]);
double or_u01(uint32_t w);
int or_init(int Ns, int Nt, int start, uint64_t seed, double *links);
void or_gauge_transform(int Ns, int Nt, double *links, uint64_t seed);
int or_heatbath_phase(int Ns, int Nt, double *links, double beta, int mu, int parity,
                      uint64_t seed, uint64_t sweep, int reverse, double creutz_below,
                      int32_t *trials_out, uint64_t *counters);
int or_heatbath_link(int Ns, int Nt, const double *links, double beta, int mu, long lex,
                     uint64_t seed, uint64_t sweep, double creutz_below, double unew[4]);
int or_update_from_staple(const double A[4], double beta, uint64_t seed, uint32_t c0,
                          uint64_t sweep, double creutz_below, double unew[4]);
int or_heatbath_link_hot(int Ns, int Nt, uint64_t init_seed, double beta, int mu, long lex,
                         uint64_t seed, uint64_t sweep, double creutz_below, double unew[4]);
void or_kp_samples(double alpha, uint64_t seed, uint64_t sweep, long n, int creutz, double *a0,
                   int32_t *trials);
double or_plaquette(int Ns, int Nt, const double *links);
double or_staple_trace_sum(int Ns, int Nt, const double *links);
void or_staple(int Ns, int Nt, const double *links, long lex, int mu, double out[4]);
double or_polyakov(int Ns, int Nt, const double *links, double *abs_mean, double *Lfield);
int or_correlator(int Ns, int Nt, const double *links, int rmax, double *out);
int or_heatbath(int Ns, int Nt, double *links, double beta, int nsweeps, uint64_t seed,
                uint64_t sweep0, double creutz_below, double *plaq_out, uint64_t *counters);

static int fail(const char *what)
{
    fprintf(stderr, "oracle sanitizer driver: %s\n", what);
    return 1;
}

static int unit_links(const double *links, long nlinks)
{
    for (long i = 0; i < nlinks; ++i) {
        const double *a = links + 4 * i;
        const double n = a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3];
        if (!(fabs(n - 1.0) < 1e-12)) return 0;
    }
    return 1;
}

static int run_lattice(int Ns, int Nt)
{
    const long V = (long)Ns * Ns * Ns * Nt;
    double *links = malloc(sizeof(double) * 16 * V);
    int32_t *trials = malloc(sizeof(int32_t) * 4 * V);
    double *plaq = malloc(sizeof(double) * 3);
    double *Lf = malloc(sizeof(double) * Ns * Ns * Ns);
    double *corr = malloc(sizeof(double) * (Ns / 2 + 1));
    uint64_t cnt[3] = {0, 0, 0};
    if (!links || !trials || !plaq || !Lf || !corr) return fail("malloc");
    if (or_init(Ns, Nt, 0, 1, links) != 0 || or_plaquette(Ns, Nt, links) != 1.0)
        return fail("cold start");
    if (or_init(Ns, Nt, 1, 2, links) != 0) return fail("hot start");
    for (int creutz = 0; creutz < 2; ++creutz) {
        const double switch_alpha = creutz ? 1.7 : 0.0;
        for (int mu = 0; mu < 4; ++mu)
            for (int p = 0; p < 2; ++p)
                or_heatbath_phase(Ns, Nt, links, 2.3, mu, p, 3, 0, (mu + p) & 1, switch_alpha,
                                  trials, cnt);
        or_heatbath(Ns, Nt, links, 0.8, 3, 4, 1, switch_alpha, plaq, cnt);
        for (int k = 0; k < 3; ++k)
            if (!isfinite(plaq[k])) return fail("plaquette");
    }
    or_heatbath(Ns, Nt, links, 0.0, 1, 5, 9, 0.0, NULL, cnt);        /* Haar branch */
    or_heatbath(Ns, Nt, links, 1e-9, 1, 5, 10, 0.0, NULL, cnt);      /* trial cap */
    if (!unit_links(links, 4 * V)) return fail("unit links");
    double u[4];
    for (long lex = 0; lex < V; lex += (V / 7) + 1)
        for (int mu = 0; mu < 4; ++mu)
            if (or_heatbath_link(Ns, Nt, links, 2.5, mu, lex, 6, 11, 0.0, u) < -1 ||
                or_heatbath_link_hot(Ns, Nt, 3, 2.5, mu, lex, 6, 0, 0.0, u) < -1)
                return fail("single link");
    double A[4];
    or_staple(Ns, Nt, links, V - 1, 3, A);
    double sa = 0.0;
    const double tr = or_staple_trace_sum(Ns, Nt, links);
    double Labs = 0.0;
    const double L = or_polyakov(Ns, Nt, links, &Labs, Lf);
    if (or_correlator(Ns, Nt, links, Ns / 2, corr) != 0) return fail("correlator");
    or_gauge_transform(Ns, Nt, links, 12);
    if (!unit_links(links, 4 * V)) return fail("gauge transform");
    for (int k = 0; k < 4; ++k) sa += A[k];
    if (!isfinite(sa) || !isfinite(tr) || !isfinite(L) || !isfinite(Labs) || !isfinite(corr[0]))
        return fail("observables");
    free(links);
    free(trials);
    free(plaq);
    free(Lf);
    free(corr);
    return 0;
}

int main(void)
{
    uint32_t ctr[4] = {0, 1, 2, 3}, key[2] = {5, 6}, out[4];
    or_philox(ctr, key, out);
    if (!(or_u01(0u) > 0.0 && or_u01(0xffffffffu) < 1.0)) return fail("u01");
    double A[4] = {0.3, -0.2, 0.5, 0.1}, u[4];
    if (or_update_from_staple(A, 2.0, 7, 3, 1, 0.0, u) < 0) return fail("staple update");
    double zero[4] = {0, 0, 0, 0};
    if (or_update_from_staple(zero, 2.0, 7, 3, 1, 0.0, u) != 0) return fail("zero staple");
    double a0[64];
    int32_t tr[64];
    or_kp_samples(3.0, 9, 2, 64, 0, a0, tr);
    or_kp_samples(0.2, 9, 2, 64, 1, a0, tr);
    const int shapes[3][2] = {{2, 2}, {4, 6}, {6, 2}};
    for (int k = 0; k < 3; ++k)
        if (run_lattice(shapes[k][0], shapes[k][1])) return 1;
    printf("oracle sanitizer driver: ok\n");
    return 0;
}
