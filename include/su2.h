/*
 * su2.h -- C ABI of the GB300 (sm_103a) SU(2) pure-gauge heat-bath library.
 *
 * The library implements the lattice part of Cardoso, Cardoso & Bicudo,
 * "Finite temperature lattice QCD with GPUs" (Excited QCD 2011):
 *   - random SU(2) start and heat-bath iterations with the mean plaquette
 *     after every iteration (Sec. 2.1, the benchmark workload);
 *   - the Polyakov loop, the order parameter of Sec. 2.2 (Eq. 1);
 *   - the Polyakov-loop correlator behind the colour-averaged free energy
 *     (Sec. 2.2, Eq. 3).
 * The paper leaves the algorithmic details to its companion paper; this
 * library fixes them as follows:
 *   - Wilson action S = beta sum_P (1 - 1/2 Re Tr U_P), beta = 4/g^2;
 *   - a link is a unit quaternion (a0,a1,a2,a3) for U = a0 + i a.sigma;
 *   - lattice extents (Ns,Ns,Ns,Nt) for (x,y,z,t), both even and >= 2,
 *     lex = x + Ns(y + Ns(z + Ns t)), parity = (x+y+z+t) mod 2;
 *   - a sweep is the eight checkerboard phases (mu, parity) in the order
 *     (0,0),(0,1),(1,0),(1,1),(2,0),(2,1),(3,0),(3,1); each link is drawn
 *     with the Kennedy-Pendleton method from its staple sum A = k Vhat,
 *     U = X Vhat^dagger, then renormalised;
 *   - all random numbers come from Philox4x32-10, key = seed, counter =
 *     (lex*4+mu, sweep, tag<<24 | trial, sweep>>32) (the direction of a new
 *     link uses the spare low bits of its first trial's block), so results are
 *     independent of launch shape, batching and graph replay, and
 *     heatbath(n) followed by heatbath(m) equals heatbath(n+m).
 *
 * Handles and memory.  A handle holds n >= 1 independent lattices (n = 1
 * for su2_lattice_create).  The library allocates NO device memory: the
 * caller queries su2_memory_requirements, allocates two device buffers
 * (any allocator; 256-byte aligned) and binds them with su2_bind_memory.
 * The buffers stay owned by the caller and must outlive the handle's use.
 * Host buffers passed to any call are owned by the caller.
 *
 * Pointers marked "host or device" may point to host memory (pageable or
 * pinned) or to device memory of the bound device; the library detects
 * which.  With a device pointer the call is asynchronous on the handle's
 * stream; with a host pointer it returns after the data has arrived.
 *
 * Test and measurement hooks (tuning-cache access, forced slab counts,
 * self-tests of the arithmetic, throughput probes for the rooflines) are
 * declared separately in su2_testing.h; they are not part of the method.
 *
 * Errors.  Every int-returning call returns SU2_OK (0) or a negative
 * status; su2_last_error() gives a message for the calling thread.  An
 * invalid argument (SU2_E_INVAL) leaves the handle unchanged.  A
 * Kennedy-Pendleton cap hit (4096 rejected trials for one link; happens
 * only for beta*k below ~1e-2) keeps that link unchanged, completes the
 * sweep and is reported as SU2_E_TRIALS by the next synchronising call
 * (su2_sync or any call that writes host memory).
 */
#ifndef SU2_GB300_H
#define SU2_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SU2_OK 0
#define SU2_E_INVAL (-1)    /* bad argument, shape or handle state */
#define SU2_E_NOMEM (-2)    /* bound buffers smaller than required */
#define SU2_E_CUDA (-3)     /* a CUDA runtime call failed */
#define SU2_E_TRIALS (-4)   /* Kennedy-Pendleton cap hit since the last sync */
#define SU2_E_BOUNDS (-5)   /* a link index out of range, caught by a build with
                               -DSU2_CHECK_BOUNDS (the access was skipped) */

#define SU2_F32 0           /* FP32 links and update, FP64 reductions */
#define SU2_F64 1           /* FP64 throughout */

#define SU2_LAYOUT_PLAIN 0  /* FP32 float4 U[mu][parity][eo]; FP64 double2
                               U[mu][parity][plane][eo], planes (a0,a1), (a2,a3) */
#define SU2_LAYOUT_PAIRS 1  /* FP32 site pairs, every Nt a multiple of 4: the
                               sites eo = q and q + V/4 of one parity (x,y,z at
                               t and t + Nt/2) share a 32-byte record
                               float4 U[mu][parity][q][2] =
                               (a0, a0', a1, a1'), (a2, a2', a3, a3') */
#define SU2_F32_PAIRS 2     /* su2_plaquette_static only: FP32 links in the
                               site-pair layout */

#define SU2_COLD 0          /* every link the identity */
#define SU2_HOT 1           /* Haar-random links (Sec. 2.1 "random SU(2)") */

typedef struct su2_lattice su2_lattice;

/* ------------------------------------------------------------------ */
/* handles                                                             */
/* ------------------------------------------------------------------ */

/* One lattice of extents Ns^3 x Nt (even, >= 2, Ns^3 Nt <= 2^30), link
 * precision dtype (SU2_F32 / SU2_F64).  *out receives the handle. */
int su2_lattice_create(int Ns, int Nt, int dtype, su2_lattice** out);

/* n independent lattices Ns[l]^3 x Nt[l] of one precision, advanced
 * together by every call (the finite-temperature scans and ensembles of
 * Sec. 2.2).  Ns, Nt: host arrays of length n, 1 <= n <= 4096. */
int su2_batch_create(int n, const int* Ns, const int* Nt, int dtype, su2_lattice** out);

/* Releases the handle (never the caller's buffers).  NULL is a no-op. */
int su2_lattice_destroy(su2_lattice* lat);

/* Number of lattices and volume V = Ns^3 Nt of lattice l. */
int su2_lattice_count(const su2_lattice* lat, int* n);
int su2_lattice_volume(const su2_lattice* lat, int l, uint64_t* V);

/* Bytes of the two device buffers a handle needs.  The link buffer holds
 * 4V links per lattice (16 B each in FP32, 32 B in FP64); the work buffer
 * holds descriptors, reduction partials, the Polyakov field, the
 * plaquette ring and a 32 MiB staging area for host transfers. */
int su2_memory_requirements(const su2_lattice* lat, size_t* link_bytes, size_t* work_bytes);

/* Device layout of the links: SU2_LAYOUT_PLAIN by default.  An SU2_F32
 * handle whose lattices all have Nt a multiple of 4 may instead store its
 * links as site pairs (SU2_LAYOUT_PAIRS): one thread of the heat bath then
 * updates the two links of a record together with packed two-lane FP32
 * instructions (the sites t and t + Nt/2 of one parity never share a
 * staple).  That issues about a third fewer instructions but needs twice
 * the registers per thread, and measured slower on every lattice from 24^4
 * to 128^4 on GB300, so it is not the default.  Both layouts take the same
 * bytes and give bit-identical links; results never depend on the layout.
 * su2_set_link_layout (before su2_bind_memory only; SU2_E_INVAL after, for
 * SU2_LAYOUT_PAIRS on an FP64 handle or on an Nt that is not a multiple of
 * 4) selects it and resets the launch shape to 0; su2_get_link_layout
 * reads it. */
int su2_set_link_layout(su2_lattice* lat, int layout);
int su2_get_link_layout(const su2_lattice* lat, int* layout);

/* Binds caller-owned device buffers of the CURRENT device (256-byte
 * aligned, at least the required sizes; SU2_E_NOMEM otherwise) and writes
 * the lattice descriptors into the work buffer (synchronous).  Links are
 * undefined until su2_init or su2_set_links.  May be called again to move
 * the handle to other buffers (contents are not copied). */
int su2_bind_memory(su2_lattice* lat, void* links, size_t link_bytes, void* work,
                    size_t work_bytes);

/* cudaStream_t (as void*) every later call is ordered on; 0 = legacy
 * default stream (the initial setting). */
int su2_set_stream(su2_lattice* lat, void* stream);

/* ------------------------------------------------------------------ */
/* the method: start, heat-bath sweeps, measurements                   */
/* ------------------------------------------------------------------ */

/* Start configuration (Sec. 2.1 "random SU(2) matrix initialization"):
 * start = SU2_COLD or SU2_HOT (Haar links, Philox tag 2 with key
 * seed + l for lattice l).  Resets each lattice's sweep counter and its
 * statistics to 0.  Asynchronous. */
int su2_init(su2_lattice* lat, int start, uint64_t seed);

/* As su2_init with one seed per lattice (host array of length n). */
int su2_batch_init(su2_lattice* lat, int start, const uint64_t* seeds);

/* nsweeps >= 0 heat-bath sweeps at coupling beta >= 0 ("100 iterations of
 * the heat bath method", Sec. 2.1).  Lattice l draws with Philox key
 * seed + l and counter field sweep = its cumulative sweep counter, which
 * advances by nsweeps.
 * plaq (nullable; host or device; double[n][nsweeps]): the mean plaquette
 * (1/6V) sum_x sum_{mu<nu} 1/2 Re Tr U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
 * after every sweep ("the calculation of the mean average plaquette at
 * each iteration", Sec. 2.1), fused into the sweep at no extra memory
 * traffic.  With plaq = NULL the fused measurement is skipped.
 * beta = 0 gives Haar links (the alpha -> 0 limit of the draw). */
int su2_heatbath(su2_lattice* lat, double beta, int nsweeps, uint64_t seed, double* plaq);

/* As su2_heatbath with one beta and one seed per lattice (host arrays of
 * length n): the temperature scan of Sec. 2.2 in one call. */
int su2_batch_heatbath(su2_lattice* lat, const double* betas, int nsweeps,
                       const uint64_t* seeds, double* plaq);

/* As su2_batch_heatbath, and after EVERY sweep the Polyakov loop (Sec. 2.2,
 * Eq. 1) and the Polyakov-loop correlator C(r), r = 0..rmax (Sec. 2.2,
 * Eq. 3), of every lattice are measured and summed in FP64 over the call's
 * sweeps: the finite-temperature scan of Sec. 2.2 (thermalise with
 * su2_batch_heatbath, then measure with this call).
 * poly_sum: host or device double[2n]: [0,n) sums of the signed spatial
 *   means of L, [n,2n) sums of their moduli.
 * corr_sum: host or device double[n][rmax+1]: sums of C(r).
 * Divide by nsweeps for the ensemble averages.  rmax <= min(Ns/2, 128). */
int su2_batch_heatbath_measure(su2_lattice* lat, const double* betas, int nsweeps,
                               const uint64_t* seeds, double* plaq, int rmax, double* poly_sum,
                               double* corr_sum);

/* Heat-bath sampler of every lattice of the handle: links whose
 * alpha = beta k is below creutz_below are drawn with Creutz's method
 * (a0 from exp(alpha a0) by inversion, accepted with sqrt(1 - a0^2);
 * acceptance ~pi/4 as alpha -> 0), the others with Kennedy-Pendleton's
 * (acceptance -> 1 as alpha grows).  0 (the default) = Kennedy-Pendleton
 * everywhere; ~1.7 is where their acceptances cross.  Both use the same
 * Philox blocks (Creutz: words 0 and 3 of trial t).  Synchronous. */
int su2_set_sampler(su2_lattice* lat, double creutz_below);

/* One checkerboard phase (mu in 0..3, parity 0/1) of every lattice at the
 * current sweep counter, which does NOT advance (the unit the sweep is
 * made of; for testing).  trials (nullable, device int32[V], n == 1
 * only) receives, at lex of every updated link, the Kennedy-Pendleton
 * trials used, 0 for a Haar draw, -1 for a cap hit. */
int su2_heatbath_phase(su2_lattice* lat, double beta, int mu, int parity, uint64_t seed,
                       int32_t* trials);

/* Mean plaquette of every lattice, out: host or device double[n]. */
int su2_plaquette(su2_lattice* lat, double* out);

/* Polyakov loop (Sec. 2.2, Eq. 1): L(x) = 1/2 Re Tr prod_{t=0}^{Nt-1}
 * U_3(x,t) and its spatial mean.  out_signed: host or device double[n],
 * the mean; out_abs (nullable): |mean|.  Also stores the field L(x) on
 * the device for su2_polyakov_correlator. */
int su2_polyakov_loop(su2_lattice* lat, double* out_signed, double* out_abs);

/* Polyakov-loop correlator (Sec. 2.2, Eq. 3; for SU(2) the traces are
 * real): C(r) = (1/(3 Ns^3)) sum_x sum_{i=x,y,z} L(x) L(x + r e_i),
 * r = 0..rmax, periodic, rmax <= min(Ns/2, 128) over the lattices.
 * Measures L first.
 * out: host or device double[n][rmax+1]; accumulate != 0 adds to out
 * (running sums over measured sweeps) instead of overwriting it. */
int su2_polyakov_correlator(su2_lattice* lat, int rmax, double* out, int accumulate);

/* ------------------------------------------------------------------ */
/* state, statistics, checkpoints                                      */
/* ------------------------------------------------------------------ */

/* Links of lattice l in the canonical layout double[V][4][4] =
 * [lex][mu][a0,a1,a2,a3] (host or device).  set rounds to FP32 for an
 * SU2_F32 handle.  Device and page-locked host buffers must be 16-byte
 * aligned (SU2_E_INVAL otherwise); the conversion kernel reads or writes
 * page-locked host memory directly, pageable host memory goes through the
 * 32 MiB staging area.  Synchronous for host pointers. */
int su2_get_links(su2_lattice* lat, int l, double* dst);
int su2_set_links(su2_lattice* lat, int l, const double* src);

/* The same in single precision: float[V][4][4], half the bytes of the
 * double layout (for SU2_F32 handles and FP32 checkpoints; an SU2_F64
 * handle rounds on get and widens on set).  Alignment, host/device and
 * synchrony as for su2_get_links / su2_set_links. */
int su2_get_links_f32(su2_lattice* lat, int l, float* dst);
int su2_set_links_f32(su2_lattice* lat, int l, const float* src);

/* U_mu(x) -> g(x) U_mu(x) g(x+mu)^+ with Haar g(x) (Philox tag 3, key
 * seed): leaves the plaquette, the Polyakov loop and the correlator
 * unchanged ("which is gauge invariant", Sec. 2.2). */
int su2_gauge_transform(su2_lattice* lat, int l, uint64_t seed);

/* Counters of lattice l since its last init: out[0] Kennedy-Pendleton
 * trials, out[1] link updates, out[2] cap hits.  Synchronous. */
int su2_stats(su2_lattice* lat, int l, uint64_t out[3]);

/* Cumulative sweep counter of lattice l (the RNG counter field);
 * checkpoint = get_links + get_sweep, resume = set_links + set_sweep. */
int su2_get_sweep(su2_lattice* lat, int l, uint64_t* sweep);
int su2_set_sweep(su2_lattice* lat, int l, uint64_t sweep);

/* ------------------------------------------------------------------ */
/* launch-shape autotuning                                             */
/* ------------------------------------------------------------------ */

/* Number of launch shapes (threads per block x minimum resident blocks per
 * SM, plain or y-slab traversal of the lattice, links per thread) compiled
 * for the phase kernel; shape 0 is the default.
 *   FP32:  0 256x4   1 128x8   2 64x16   3 32x32   4 256x4 slab  5 128x8 slab
 *          6 32x32 /2  7 32x32 /4  8 32x32 /8  9 32x16 /4 staged
 *          10 32x32 /2 P  11 32x32 /1 P  12 32x32 slab /8  13 32x32 slab /16
 *   FP64:  0 256x1   1 128x4   2 64x8   3 64x4   4 32x16   5 32x8
 *          6 32x16 /2  7 32x16 /4  8 32x16 /8  9 32x16 /16  10 64x8 G8
 *          11 32x16 G8  12 32x16 /2 P  13 32x16 /8 P
 *   FP32 site pairs (SU2_LAYOUT_PAIRS; R counts pairs): 0 256x2  1 32x16
 *          2 32x20  3 32x24  4 32x28  5 32x16 /2  6 32x20 /2  7 32x24 /2
 *          8 32x24 /4  9 32x20 /4  10 32x24 /1 P  11 32x16 /1 P
 *          12 32x24 slab /4  13 32x16 slab /4
 * (/R: R links per thread with a per-warp queue of rejected Kennedy-
 * Pendleton trials, retried 32 at a time; slab: large lattices walked in y
 * slabs so the +-t neighbours stay in L2; P, persistent: on a single
 * lattice only the blocks that fit on the GPU at once are launched, each
 * walking tiles of R rounds in grid-stride order with one queue drain at
 * the end; on a batch one block per tile, as the other shapes; staged: the
 * neighbour rows of a warp copied into shared memory by bulk copies; G8:
 * eight lanes per link, the staple terms and trials in parallel, for small
 * FP64 lattices.)  Small blocks spread tiny lattices over more SMs; several
 * links per thread pay off on large ones.  Results never depend on the
 * shape (the random streams are keyed by link and sweep). */
#define SU2_NUM_LAUNCH_CONFIGS 14

/* Launch index SU2_LAUNCH_CLUSTER (one past the shapes): a whole sweep in
 * ONE launch of one thread-block cluster (up to 16 CTAs on 16 SMs) that
 * holds all links of the lattice in its distributed shared memory, the
 * eight phases separated by the hardware cluster barrier.  For one FP32
 * lattice in the plain layout whose links fit the cluster's shared memory
 * (8^4, 10^4, 12^4, ...: Vh = V/2 divisible by the cluster size and
 * 8 Vh/S links of 16 B per CTA); elsewhere su2_set_launch_config refuses it
 * with SU2_E_INVAL, and su2_autotune times it only where it applies.  The
 * links are bit-identical to the shapes'; the single-phase entry point
 * (su2_heatbath_phase) keeps using the last shape. */
#define SU2_LAUNCH_CLUSTER 14

/* Times every launch shape on this handle's lattices (whole sweeps with the
 * fused plaquette, replayed as in su2_heatbath, ~20 ms per shape in each of
 * three interleaved rounds, best round kept) and keeps the fastest.
 * OVERWRITES the links: on return every lattice holds the hot start of
 * su2_init(SU2_HOT, 0x5EED) with zeroed counters; call it before su2_init
 * or su2_set_links.  If the environment variable SU2_AUTOTUNE_CACHE names
 * a file, the choice is appended there under a key made of the GPU name,
 * the precision and link layout, the lattice shapes, the shape table and
 * the coupling band, and su2_bind_memory of any later handle with the same
 * key (at beta = 2.4) starts with the cached shape.
 * chosen (nullable): the index picked.  Synchronous. */
int su2_autotune(su2_lattice* lat, int* chosen);

/* As su2_autotune, timed at the couplings the handle will run: betas is a
 * host array of n values (NULL: beta = 2.4 for every lattice, which is what
 * su2_autotune does).  The retry queue's share of the work follows the
 * Kennedy-Pendleton acceptance, which depends on beta, so the best shape
 * can differ between couplings.  The cache key carries the coupling band
 * floor(2 log2 mean(beta)); with SU2_AUTOTUNE_CACHE set, a choice cached
 * for the same GPU, shapes and band is taken without timing (the links are
 * still left in the tuning seed's hot start). */
int su2_autotune_beta(su2_lattice* lat, const double* betas, int* chosen);

/* Select a launch shape by index (0 .. SU2_NUM_LAUNCH_CONFIGS-1, or
 * SU2_LAUNCH_CLUSTER once memory is bound) / read the current one with its
 * threads per block and minimum blocks per SM (for the cluster sweep: the
 * threads per CTA and the CTAs in the cluster). */
int su2_set_launch_config(su2_lattice* lat, int cfg);
int su2_get_launch_config(const su2_lattice* lat, int* cfg, int* threads, int* min_blocks);

/* Waits for the handle's stream; returns SU2_E_TRIALS (once) if a cap hit
 * occurred since the previous synchronising call. */
int su2_sync(su2_lattice* lat);

/* Message of the last failing call on this thread ("" if none). */
const char* su2_last_error(void);

/* ------------------------------------------------------------------ */
/* allocation-free measurement                                          */
/* ------------------------------------------------------------------ */

/* Largest lattice (sites) su2_plaquette_static accepts. */
#define SU2_STATIC_MAX_SITES 16777216

/* The mean plaquette of one lattice, computed without any device
 * allocation and without a caller work buffer.  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory,
 * such as code running inside a host framework that owns the whole device
 * pool (its own cudaMalloc would fail or break the framework's budget), or
 * code that must avoid the device-wide synchronisation that cudaMalloc and
 * cudaFree can cause.
 * links: device memory of the CURRENT device holding one lattice in the
 *   library's link layout -- the link buffer of a single-lattice handle
 *   (FP32: float4 U[mu][parity][eo]; FP64: double2 U[mu][parity][plane][eo],
 *   plane 0 = (a0,a1), plane 1 = (a2,a3); eo = lex >> 1).
 * dtype: SU2_F32 or SU2_F64 for those layouts, SU2_F32_PAIRS for FP32 links
 *   in the site-pair layout (SU2_LAYOUT_PAIRS; Nt a multiple of 4): pass
 *   SU2_F32_PAIRS for a handle whose su2_get_link_layout gives it.
 * Ns, Nt: even, >= 2, Ns^3 Nt <= SU2_STATIC_MAX_SITES (else SU2_E_INVAL).
 * out: host or device double; a host output makes the call synchronous.
 * stream: cudaStream_t (as void*), 0 = legacy default stream.
 * Scratch: a fixed 512 KiB array in the library's static device memory,
 * held by every GPU that loads the library until the process exits.  The
 * first call on each device looks up that array's device address (with
 * cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the array and it keeps the last call's contents: calls
 * whose work overlaps on the GPU (other streams or host threads) race on
 * it and must be ordered by the caller.  Allocates nothing. */
int su2_plaquette_static(const void* links, int Ns, int Nt, int dtype, double* out,
                         void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SU2_GB300_H */
