// su2_internal.h -- data structures shared by the kernels and the C-ABI
// layer of the SU(2) heat-bath library.
//
// Memory model: the caller owns two device buffers and binds them to a
// handle.  The LINK buffer holds every lattice of the handle; the WORK
// buffer holds the per-lattice descriptors, reduction partials, the
// per-sweep plaquette ring, the Polyakov field and a staging area for host
// copies.  The library never allocates device memory.
//
// Link layout of one lattice (V sites, Vh = V/2):
//   FP32: float4   U[mu][parity][eo]              (16 B per link)
//   FP64: double2  U[mu][parity][plane][eo]       plane 0 = (a0,a1), 1 = (a2,a3)
// so a warp touching 32 consecutive eo reads 512 contiguous bytes per access.
//   FP32 site pairs (Nt a multiple of 4): the sites eo = q and q + Vh/2 (the
//   same x, y, z at t and t + Nt/2, of the same parity) share one 32 B record
//   float4 U[mu][parity][q][2] = (a0, a0', a1, a1'), (a2, a2', a3, a3'), so
//   one load gives both links' components side by side, the operand layout
//   of the packed two-lane FP32 instructions (FFMA2/FMUL2/FADD2).
#pragma once
#include <cstddef>
#include <cstdint>

#include "su2_device.cuh"

namespace su2 {

constexpr int TPB = 256;            // threads per block of the non-phase kernels

// Launch shapes of the phase kernel the autotuner chooses from (threads per
// block, minimum resident blocks per SM); entry 0 is the default.  Row 0:
// FP32, row 1: FP64, row 2: FP32 site pairs.
// slab: walk large lattices in y slabs (EoSite::from_slab) -- FP32 only,
// since the FP64 kernel is bound by its arithmetic, not by re-reads.
// rounds: links per thread; above 1 the kernel with the per-warp retry
// queue (hb_phase_queue_kernel) runs.
// persistent (single-lattice handles): only the blocks that fit on the GPU
// at once are launched, and each walks tiles of R rounds in grid-stride
// order, so its retry queue carries over from tile to tile and drains once.
// group (FP64): lanes per link; above 1 the cooperative kernel runs, whose
// G lanes share one link's staple terms and try several Kennedy-Pendleton
// trials at once (small lattices, where the FP64 work of few links per warp
// sets the time).
// stage (FP32 queued kernel, lattices with Nh = 32): each round one lane
// brings the 18 neighbour rows of the warp's 32 sites into shared memory
// with bulk copies (cp.async.bulk behind an mbarrier), and the lanes read
// their neighbours there.
struct LaunchCfg {
    int threads, min_blocks;
    bool slab;
    int rounds;
    bool persistent;
    int group = 1;
    bool stage = false;
};
constexpr int NUM_LAUNCH_CFG = 14;
// rows of the table: link layouts with their own phase kernels
constexpr int ROW_F32 = 0, ROW_F64 = 1, ROW_F32_PAIRS = 2, NUM_ROWS = 3;
// Small blocks (64, 32 threads) spread tiny lattices over more SMs; several
// links per thread pay off on large lattices (one queue pass retries 32
// rejected trials at once) but leave small ones with too few blocks.
constexpr LaunchCfg LAUNCH_CFG[NUM_ROWS][NUM_LAUNCH_CFG] = {
    {{256, 4, false, 1, false}, {128, 8, false, 1, false}, {64, 16, false, 1, false},
     {32, 32, false, 1, false}, {256, 4, true, 1, false}, {128, 8, true, 1, false},
     {32, 32, false, 2, false}, {32, 32, false, 4, false}, {32, 32, false, 8, false},
     {32, 16, false, 4, false, 1, true}, {32, 32, false, 2, true}, {32, 32, false, 1, true},
     {32, 32, true, 8, false}, {32, 32, true, 16, false}},
    {{256, 1, false, 1, false}, {128, 4, false, 1, false}, {64, 8, false, 1, false},
     {64, 4, false, 1, false}, {32, 16, false, 1, false}, {32, 8, false, 1, false},
     {32, 16, false, 2, false}, {32, 16, false, 4, false}, {32, 16, false, 8, false},
     {32, 16, false, 16, false}, {64, 8, false, 1, false, 8}, {32, 16, false, 1, false, 8},
     {32, 16, false, 2, true}, {32, 16, false, 8, true}},
    // FP32 site pairs: one thread updates two links (t and t + Nt/2) per
    // round with packed two-lane arithmetic; `rounds` counts pairs
    {{256, 2, false, 1, false}, {32, 16, false, 1, false}, {32, 20, false, 1, false},
     {32, 24, false, 1, false}, {32, 28, false, 1, false}, {32, 16, false, 2, false},
     {32, 20, false, 2, false}, {32, 24, false, 2, false}, {32, 24, false, 4, false},
     {32, 20, false, 4, false}, {32, 24, false, 1, true}, {32, 16, false, 1, true},
     {32, 24, true, 4, false}, {32, 16, true, 4, false}},
};
static_assert(NUM_LAUNCH_CFG % 2 == 0, "shapes compile in pairs");
// largest y-slab window (sites between a site and its t neighbour, times
// the bytes a site's update touches) kept in L2
constexpr double SLAB_WINDOW_BYTES = 8.0 * (1 << 20);

constexpr int KP_CAP = 4096;        // Kennedy-Pendleton trial cap
constexpr int PLAQ_RING = 4096;     // per-lattice plaquette slots for host output
constexpr size_t STAGE_BYTES = size_t(32) << 20;
constexpr uint32_t STATUS_CAP_HIT = 1u;
constexpr uint32_t STATUS_BOUNDS = 2u;  // bounds-checked builds only
constexpr uint32_t STATUS_STAGE = 4u;   // a bulk copy of neighbour rows did not arrive in time
constexpr int SWEEP_CHUNK = TPB * 8;   // plaquette partials summed per sweep_end block
constexpr int MAX_RMAX = 128;          // largest correlator separation
constexpr int TRIAL_SLOTS = 64;        // per-lattice trial counters (spread atomics)

// One per lattice, resident in the work buffer.  The first block is fixed
// at bind time; the second is written by the parameter kernel at every
// heat-bath call; the counters are advanced by the kernels.
struct LatDesc {
    int32_t Ns, Nt, Nh, Vs;
    uint32_t V, Vh;
    FastDiv div_nh, div_ns;
    int32_t ysplit, Ny;     // y slabs of the large-lattice traversal, Ny = Ns / ysplit
    FastDiv div_ny, div_nt;
    FastDiv div_nt2;        // Nt / 2: the t extent of the lattice of site pairs
    int32_t paired;         // FP32 links stored as site pairs (t, t + Nt/2)
    uint32_t Vq;            // site pairs per parity (Vh / 2) when paired
    double creutz_below;    // alpha below which Creutz's draw replaces Kennedy-Pendleton's
    float creutz_below_f;
    const double2* fp64_table;  // the FP64 path's log and sin/cos tables (work memory)
    uint64_t link_off;      // byte offset of this lattice in the link buffer
    uint64_t field_off;     // double offset of its Polyakov field
    // per call
    double beta;
    float beta_f;           // beta rounded once for the FP32 kernels
    float half_inv_beta_f;  // 1 / (2 beta) rounded once: 1 / (2 alpha) = half_inv_beta_f / k
    double half_inv_beta;   // 1 / (2 beta) for the FP64 kernels: 1 / (2 alpha) = half_inv_beta / k
    uint64_t seed;
    uint64_t sweep_base;    // sweep index stored at plaq_out[0]
    double* plaq_out;       // device, nullable
    // advanced by the kernels
    uint64_t sweep;         // cumulative sweep counter
    unsigned long long trials, updates, caps;
};

// Everything a kernel needs, passed by value.
struct Ctx {
    void* links;
    LatDesc* desc;
    const uint32_t* phase_start;   // [n+1] first block of each lattice, V/2 links
    const uint32_t* site_start;    // [n+1] ... V sites
    const uint32_t* spat_start;    // [n+1] ... Ns^3 spatial sites
    double* plaq_partial;          // [3][phase blocks * warps per block], per warp
    double* obs_partial;           // [obs_rows][max(site, spat) blocks]
    double* field;                 // Polyakov fields
    double* ring;                  // [n][PLAQ_RING]
    double* chunk_partial;         // [n][max_chunks] sweep_end chunk sums
    uint32_t* chunk_count;         // [n] sweep_end tickets (zero between sweeps)
    unsigned long long* trial_slots;  // [n][TRIAL_SLOTS] Kennedy-Pendleton trial counts
    uint32_t* status;
    int n;
    uint32_t phase_blocks, site_blocks, spat_blocks;
    uint32_t max_chunks;
    uint32_t phase_wpb;            // warps per phase block of this launch shape
};

// first grid block of lattice l; lattice 0 starts at block 0, so a single
// lattice's kernels need no load (one global-memory round trip fewer before
// the first link load)
__device__ __forceinline__ uint32_t first_block(const uint32_t* start, int l)
{
    return l == 0 ? 0u : __ldg(start + l);
}

// lattice owning grid block b: largest l with start[l] <= b
__device__ __forceinline__ int lattice_of_block(const uint32_t* start, int n, uint32_t b)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(start + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ----- launchers (defined in the .cu files, called by the C-ABI layer) -----
constexpr int PARAM_CHUNK = 64;
struct ParamChunk {
    int first, count;
    double beta[PARAM_CHUNK];
    uint64_t seed[PARAM_CHUNK];
    double* plaq_out[PARAM_CHUNK];
};
cudaError_t launch_set_params(const Ctx& c, const ParamChunk& pc, cudaStream_t s);
// hybrid: compile-time variant with Creutz's draw below each lattice's
// creutz_below (the plain variant never looks at it)
cudaError_t launch_phase(const Ctx& c, int row, int cfg, int mu, int parity, bool plaq,
                         int32_t* dbg_trials, bool hybrid, cudaStream_t s);
cudaError_t launch_sweep_end(const Ctx& c, bool plaq, cudaStream_t s);

// the tables of the FP64 path's logarithm and sine/cosine (ln_u01_tab,
// sincospi_tab, su2_math.cuh: layout TAB_*), filled on the host
void fill_fp64_table(double2* tab);

// The whole sweep of a small single FP32 lattice in one thread-block
// cluster (cluster.cu): launch index NUM_LAUNCH_CFG.
constexpr int CFG_CLUSTER = NUM_LAUNCH_CFG;
constexpr int CLUSTER_MAX = 16;  // CTAs per cluster (16 needs the non-portable opt-in)
struct ClusterGeom {
    int S = 0;          // CTAs in the cluster
    uint32_t C = 0;     // links per (mu, parity) per CTA: Vh / S
    FastDiv div_c{};
    int threads = 0;    // per CTA
    size_t smem = 0;    // dynamic shared memory per CTA
};
bool cluster_geometry(uint32_t Vh, int dtype_f32, int n, ClusterGeom* g);
bool cluster_launchable(const ClusterGeom& g);
cudaError_t launch_cluster_sweep(const Ctx& c, const ClusterGeom& g, bool plaq, bool hyb,
                                 cudaStream_t s);
cudaError_t launch_init(const Ctx& c, int dtype, int l, uint32_t V, int hot, uint64_t seed,
                        cudaStream_t s);
// canonical values in double (cdtype 1) or float (cdtype 0); pairs_whole:
// the whole lattice (lex0 = 0, nsite = V) of a lattice stored as FP32 site
// pairs, converted record by record
cudaError_t launch_links_to_canonical(const Ctx& c, int dtype, int l, uint32_t lex0,
                                      uint32_t nsite, void* dst, int cdtype, cudaStream_t s,
                                      bool pairs_whole = false);
cudaError_t launch_links_from_canonical(const Ctx& c, int dtype, int l, uint32_t lex0,
                                        uint32_t nsite, const void* src, int cdtype,
                                        cudaStream_t s, bool pairs_whole = false);
cudaError_t launch_gauge(const Ctx& c, int dtype, int l, uint32_t V, uint64_t seed, cudaStream_t s);
cudaError_t launch_plaquette(const Ctx& c, int dtype, double* out_dev, cudaStream_t s);
cudaError_t launch_polyakov(const Ctx& c, int dtype, double* out_signed_dev,
                            double* out_abs_dev, int accumulate, cudaStream_t s);
cudaError_t launch_correlator(const Ctx& c, int dtype, int rmax, double* out_dev, int accumulate,
                              cudaStream_t s);

// sets the message returned by su2_last_error() for the calling thread
void record_error(const char* msg);

}  // namespace su2
