/*
 * su2_testing.h -- test and measurement hooks of the SU(2) heat-bath
 * library (libsu2gb300.so), kept apart from the method's boundary in su2.h.
 *
 * None of these calls is part of the paper's method.  They exist so that
 * the test-suite can reach host-side logic (the tuning cache, forced slab
 * counts, the exact division used for site indexing), check the FP32
 * transcendental forms exhaustively, and so that the benchmark can measure
 * the arithmetic rooflines' denominators on the GPU it runs on.
 * Return values follow su2.h: SU2_OK (0) or a negative SU2_E_* status.
 */
#ifndef SU2_GB300_TESTING_H
#define SU2_GB300_TESTING_H

#include "su2.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ */
/* launch-shape tuning cache and traversal                             */
/* ------------------------------------------------------------------ */

/* The handle's tuning-cache key: GPU name | precision | lattice count |
 * total volume | hash of the lattice shapes | hash of the launch-shape
 * table.  buf receives a NUL-terminated string of at most len bytes
 * (SU2_E_INVAL if it does not fit). */
int su2_tune_key(const su2_lattice* lat, char* buf, size_t len);

/* Lookup in / append to a tuning-cache file ("key cfg ms" per line, later
 * lines win).  Lookup returns 1 if the key is found (*cfg set), 0 if not;
 * store returns SU2_OK or SU2_E_INVAL (bad shape index, unwritable file). */
int su2_tune_cache_lookup(const char* path, const char* key, int* cfg);
int su2_tune_cache_store(const char* path, const char* key, int cfg, double ms);

/* Walk every lattice in S y-slabs under the slab launch shapes (S must
 * divide every Ns; by default S is chosen from the lattice size so that
 * the +-t neighbour window stays within 8 MB of L2).  Synchronous. */
int su2_set_slabs(su2_lattice* lat, int S);

/* ------------------------------------------------------------------ */
/* self-tests of the arithmetic                                        */
/* ------------------------------------------------------------------ */

/* Exhaustive check, over every uniform grid point u = (k + 1/2) 2^-23, of
 * the FP32 forms the heat-bath draw uses against FP64 references.
 * out: device double[4] receiving the maximum relative error of ln u, the
 * maximum absolute error of cos^2(2 pi u), of sin/cos(2 pi u), and the
 * maximum relative error of sqrt(u).  Asynchronous on `stream`. */
int su2_selftest_math(void* out, void* stream);

/* Host-side exact division used for site indexing: returns the number of
 * n in [0, limit) and divisors 1..dmax for which it differs from n / d. */
uint64_t su2_selftest_fastdiv(uint32_t dmax, uint32_t limit);

/* ------------------------------------------------------------------ */
/* throughput probes (roofline denominators)                           */
/* ------------------------------------------------------------------ */

/* FMA throughput of the current device in FP32 (dtype SU2_F32) or FP64
 * (SU2_F64): a grid of 8 blocks of 256 threads per SM, each thread running
 * 8 independent FMA chains of `iters` steps, launched twice on `stream`
 * and the second launch timed with CUDA events.  *fma_per_s: FMA
 * instructions per second summed over all threads (one FMA = 2 flops).
 * Synchronous; allocates nothing. */
int su2_probe_fma_rate(int dtype, int iters, double* fma_per_s, void* stream);

/* Throughput of one FP64 math function of the heat-bath draw, as the
 * library calls it: fn = SU2_PROBE_LOG (log), SU2_PROBE_COSPI (cospi),
 * SU2_PROBE_SINCOSPI (sincospi, both results), SU2_PROBE_SQRT (sqrt),
 * SU2_PROBE_RSQRT (rsqrt).  Same grid and timing as su2_probe_fma_rate:
 * each thread runs 8 independent chains of `iters` calls, each call fed by
 * the previous one's result (log(x + 2), cospi(x), sincospi(x) summed,
 * sqrt(x), rsqrt(x): arguments stay in the functions' ordinary range).
 * *calls_per_s: calls per second summed over all threads (the one add of
 * the log and sincospi chains is included).  Synchronous; allocates
 * nothing. */
#define SU2_PROBE_LOG 0
#define SU2_PROBE_COSPI 1
#define SU2_PROBE_SINCOSPI 2
#define SU2_PROBE_SQRT 3
#define SU2_PROBE_RSQRT 4
/* SU2_PROBE_LN_TABLE: the FP64 heat bath's own logarithm of a uniform,
 * table-driven (the argument's bits give the uniform; chains feed each
 * result's low bits back in) */
#define SU2_PROBE_LN_TABLE 5
/* SU2_PROBE_COS_TABLE / SU2_PROBE_SINCOS_TABLE: its table-driven cosine
 * (the trials' cos(2 pi r2)) and sine + cosine (the direction's angle) of
 * the grid values */
#define SU2_PROBE_COS_TABLE 6
#define SU2_PROBE_SINCOS_TABLE 7
int su2_probe_special_rate(int fn, int iters, double* calls_per_s, void* stream);

/* The FP64 heat bath's table-driven logarithm against CUDA's log on all
 * 2^23 uniforms u = (2k + 1) 2^-24 it is used on.  out: device buffer of 2
 * doubles, filled on `stream` with the largest absolute difference and the
 * largest difference in units of the last place of CUDA's result.  Uploads
 * the table (synchronous); the kernel is asynchronous on `stream`. */
int su2_selftest_ln(void* out, void* stream);

/* The FP64 heat bath's table-driven sine and cosine of pi y against CUDA's
 * sincospi: out (device, 2 doubles) gets the cosine's largest absolute
 * difference over the trials' 2^23 arguments y = (2k + 1) 2^-23 and the
 * sine's and cosine's over the direction's 2^18 arguments
 * y = (2k + 1) 2^-18.  Uploads the table (synchronous); the kernel is
 * asynchronous on `stream`. */
int su2_selftest_trig(void* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SU2_GB300_TESTING_H */
