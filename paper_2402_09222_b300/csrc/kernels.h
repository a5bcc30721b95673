// kernels.h -- internal kernel-launch interface between the C-ABI layer
// (mcx_api.cu) and the kernel translation units.  Not part of the public ABI.
#pragma once

#include <cmath>

#include "mcx_internal.cuh"

namespace mcx {

// ---------------------------------------------------------------- lookups
int launch_xs_lookup_exact(const Tables& t, int64_t n, const double* E, const int32_t* mat,
                           const int32_t* perm, double* out, int grid, cudaStream_t st);
// resident 256-thread blocks per SM of the fast lookup (its register cap)
constexpr int kFastBlocksPerSm = 4;
// the same for the round-linear form (MCX_LOOKUP_LINEAR)
constexpr int kLinBlocksPerSm = 3;
// work: a device counter for in-order chunked scheduling of binned orders
// (zeroed by the launch), or nullptr for a grid-stride loop.  linear: on a
// binned order with a work counter, the round-linear sums (within the fast
// bound, not bit-identical to the per-lookup sums).  inputs_binned: E and mat
// are given in the processing order (lookup j has E[j], mat[j] and writes
// row perm[j]); binned orders with a work counter only.
int launch_xs_lookup_fast(const Tables& t, int64_t n, const double* E, const int32_t* mat,
                          const int32_t* perm, void* out, bool out32, int grid, cudaStream_t st,
                          unsigned long long* work = nullptr, bool linear = false, bool inputs_binned = false);
struct SortParams {
    int32_t n_materials = 1;
    int32_t n_ebuckets = 1;
    float ln_lo = 0.f, scale = 0.f;  // bucket = (ln E - ln_lo) * scale
};

// Lookups per (material, log-energy bucket) the binning of a lookup batch
// aims at on average.  A warp's 64-lookup round then spans one or two
// buckets, so the fewer grid points a bucket holds, the fewer species'
// bracketing intervals a round straddles; finer buckets leave rounds spanning
// several.  1e8 lookups, two-level binning: 96 / 112 / 128 / 160 / 192 per
// bucket give 24.07 / 23.92 / 23.89 / 24.21 / 24.13 ms per step (the last two
// on different boxes: 128 and 160 gave 24.21 where 192 gave 24.40).
#ifndef MCX_LOOKUPS_PER_BUCKET
#define MCX_LOOKUPS_PER_BUCKET 128
#endif
constexpr int64_t kLookupsPerBucket = MCX_LOOKUPS_PER_BUCKET;

// The same for the binned backward, whose warps take 32 lookups at a time
// and gain from the narrowest energy span per warp (measured best at 8).
#ifndef MCX_BACKWARD_LOOKUPS_PER_BUCKET
#define MCX_BACKWARD_LOOKUPS_PER_BUCKET 8
#endif
constexpr int64_t kBackwardLookupsPerBucket = MCX_BACKWARD_LOOKUPS_PER_BUCKET;

// Buckets per material of a lookup batch at least: below n = materials x
// per_bucket x this, a warp's 64 lookups span several grid intervals however
// fine the buckets, and finer buckets cost little at that size (1e8 lookups
// from host buffers in 4M-lookup chunks with FP32 outputs: 43.2 ms against
// 49.9 ms at n / (materials x 192) buckets).
#ifndef MCX_MIN_LOOKUP_EBUCKETS
#define MCX_MIN_LOOKUP_EBUCKETS 16384
#endif
// Binning parameters of a batch of n lookups over n_materials materials with
// energies in [emin, emax]: n / (n_materials * per_bucket) buckets per
// material, at least MCX_MIN_LOOKUP_EBUCKETS, at most max_bins bins in all
// (and at least 1 bucket).
inline SortParams lookup_sort_params(int n_materials, double emin, double emax, int64_t n, int64_t max_bins,
                                     int64_t per_bucket = kLookupsPerBucket)
{
    SortParams sp;
    sp.n_materials = n_materials;
    int64_t nb = n / ((int64_t)n_materials * per_bucket);
    if (nb < MCX_MIN_LOOKUP_EBUCKETS) nb = MCX_MIN_LOOKUP_EBUCKETS;
    if (nb > max_bins / n_materials) nb = max_bins / n_materials;
    sp.n_ebuckets = nb < 1 ? 1 : (int32_t)nb;
    sp.ln_lo = (float)std::log(emin);
    sp.scale = (float)((double)sp.n_ebuckets / (std::log(emax) - std::log(emin)));
    return sp;
}

// The TMA-staged form of the binned fast lookup (perm and work required; err
// receives 1 if a bounded wait ran out).  Returns -2 when a material is too
// large for a stage (use launch_xs_lookup_fast), -1 on a launch error.
int launch_xs_lookup_staged(const Tables& t, const SortParams& sp, int64_t n, const double* E,
                            const int32_t* mat, const int32_t* perm, void* out, bool out32, int sm_count,
                            cudaStream_t st, unsigned long long* work, unsigned int* err);
int launch_xs_indices(const Tables& t, int64_t n, const double* E, const int32_t* mat,
                      int32_t max_species, int32_t* kout, int grid, cudaStream_t st);
int launch_build_hash(const Tables& t, int32_t* hidx, int grid, cudaStream_t st);
// Per interval and channel (s[k+1] - s[k]) / (g[k+1] - g[k]) from the device
// sigma table (0 at a species' last point), into slope [n_points][n_ch]; and
// per point the total t = s_scatter + s_absorb with its slope into ttot
// (libraries with the transport's channels, else zeros).
int launch_build_slopes(const Tables& t, double* slope, double2* ttot, int grid, cudaStream_t st);
// The transport's per-point values (grid energy, total, absorption, nu-
// fission and their slopes, from E, ttot, slope and sigma) as FP32 pairs into
// tpair [n_points][t.tpair_w], and the nnz densities as pairs into mden2.
int launch_build_pairs(const Tables& t, float4* tpair, float2* mden2, int64_t nnz, int grid, cudaStream_t st);
// Widest hash window (in grid points, window end inclusive) into *out (device int).
int launch_hash_max_window(const Tables& t, int32_t* out, int grid, cudaStream_t st);
int launch_xs_backward(const Tables& t, int64_t n, const double* E, const int32_t* mat,
                       const double* grad_out, double* grad_dens, double* grad_sigma, int grid,
                       cudaStream_t st);
// The same adjoint over a binned order perm (lookups sorted by material and
// log-energy bucket): warps of one material aggregate their contributions
// per species and grid interval before the atomics (nnz material entries;
// work: a chunk counter, zeroed by the launch).
int launch_xs_backward_binned(const Tables& t, int64_t nnz, int64_t n, const double* E, const int32_t* mat,
                              const int32_t* perm, const double* grad_out, double* grad_dens,
                              double* grad_sigma, int sm_count, unsigned long long* work, cudaStream_t st);
int launch_update_tables(const Tables& t, const double* dens_src, int64_t nnz, double* mden,
                         int4* ment, const double* sig_src, void* sigma, float4* frec,
                         cudaStream_t st);
int launch_debug_neg_log(const double* x, int64_t n, double* out, cudaStream_t st);
int launch_debug_transport_xs(const Tables& t, int64_t n, const double* E, const int32_t* mat, float2* cum2,
                              int64_t stride, double* out, cudaStream_t st);
int launch_debug_uniforms(uint2 key, uint64_t hist, uint32_t first, int64_t n, double* out,
                          cudaStream_t st);

// Counting sort of lookups by key = material * n_ebuckets + log-energy bucket.
// Scratch: bins [n_materials * n_ebuckets + 1 + kSortScanParts] uint32 (the
// counters, then the part sums of the multi-block scan).  perm receives the
// lookup indices in bin order.
constexpr int kSortScanParts = 1024;
int launch_lookup_sort(const SortParams& sp, int64_t n, const double* E, const int32_t* mat,
                       uint32_t* bins, int32_t* perm, int grid, cudaStream_t st);

// The same binning in two levels (coarse bins of 512 consecutive bins,
// counted per tile of 16384 lookups in shared memory; then each coarse bin sorted
// by its fine bins in shared memory): no global atomic per lookup.  Scratch:
// place [lookup_sort2_place_words] uint32, keys [n] uint32, tidx [n] int32,
// tfine [n] uint16.
// Returns -2 when the batch's tiles x coarse bins exceed 2^28 (above 1e9
// lookups; use launch_lookup_sort), -1 on a launch error.
#ifndef MCX_BIN2_MIN_LOOKUPS
#define MCX_BIN2_MIN_LOOKUPS (1 << 22)
#endif
constexpr int64_t kBin2MinLookups = MCX_BIN2_MIN_LOOKUPS;   // batches from this size take it
size_t lookup_sort2_place_words(const SortParams& sp, int64_t n);
// With a carry, every lookup's energy follows its index through both passes
// (coarse-order scratch tE [n] double) into the binned order, and its
// material is taken from its bin: Eb[j] = E[perm[j]], Mb[j] = mat[perm[j]]
// (-1 for a material id outside [0, n_materials)).
struct Bin2Carry {
    double* tE;
    double* Eb;
    int32_t* Mb;
};
int launch_lookup_sort2(const SortParams& sp, int64_t n, const double* E, const int32_t* mat, uint32_t* place,
                        uint32_t* keys, int32_t* tidx, uint16_t* tfine, int32_t* perm, int sm_count,
                        cudaStream_t st, const Bin2Carry* carry = nullptr);
// Eb[j] = E[perm[j]], Mb[j] = mat[perm[j]] by a gather (-1 for a material
// id outside [0, n_materials); NaN and -1 for an index outside [0, n)).
int launch_gather_inputs(int64_t n, const int32_t* perm, const double* E, const int32_t* mat, int n_materials,
                         double* Eb, int32_t* Mb, int grid, cudaStream_t st);

// First failed bounds check of each kernel translation unit since the last
// read (site << 56 | index; 0: none), cleared by the read; always 0 in
// release builds.
unsigned long long bounds_error_xs_exact();
unsigned long long bounds_error_xs_fast();
unsigned long long bounds_error_transport();
unsigned long long bounds_error_adjoint();

// Tables, FP32 densities and binning parameters of a loaded problem, for
// entry points defined outside the C-ABI translation unit.
struct LookupView {
    Tables tables;
    SortParams sort;
    int device = 0;
    int grid = 0;
    int sm_count = 0;
    double emin = 0.0, emax = 0.0;   // energy range of the binning
};

}  // namespace mcx
struct mcx_problem;
namespace mcx {
int problem_lookup_view(const mcx_problem* p, LookupView* v);
int set_error(int code, const char* msg);

// ------------------------------------------------------------- transport
enum : uint8_t {
    PF_ALIVE = 1,
    PF_NEED_XS = 2,
    PF_INPIN = 4,
    PF_COLLIDE = 8,
    PF_RETIRED = 16,
};

enum { OUT_ABSORBED = 0, OUT_LEAK_XHI = 1, OUT_LEAK_OTHER = 2, OUT_CUTOFF = 3, OUT_COLLISIONS = 4,
       N_OUT = 5 };

// A fission site: position, lattice cell (ci * n + cj) and inside-pin flag.
struct FissionSite {
    double x, y, z;
    int32_t cell;
    int32_t inpin;
};

// Per-generation device accumulators of an eigenvalue run.
struct EigenCtl {
    double k_col;                  // sum of nuSigma_f / Sigma_t over collisions
    double k_tl;                   // sum of d nuSigma_f over flights
    unsigned long long banked;     // sites banked (may exceed the bank capacity)
    unsigned long long pad;
};

// One transport problem as the kernels see it (device array, one per
// problem of a run).
struct ProblemDev {
    int32_t geometry;
    int32_t lattice_n;
    int32_t nb;          // tally bins
    int32_t n_batches;
    int32_t n_ebins;
    int32_t M;           // materials with derivative tallies (0 = off)
    double pitch, radius, height, slab_length, half, E0, E_cut;
    double radius2;      // radius * radius (the same product the flight would form)
    const int32_t* region_material;
    const double* lat_plane;   // lattice: x (and y) of cell plane i = -half + pitch i, i = 0..n
    const double* lat_centre;  // lattice: centre of cell i = -half + pitch (i + 1/2)
    const double* ebin_edges;
    uint2 key;            // Philox key (seed, problem id)
    int64_t n_hist_total; // defines batches
    int64_t first;        // first history of this run
    double* flux;
    double* absorb;
    double* outcome;
    double* dflux;
    double* dabsorb;
    double* doutcome;
    uint32_t* ncoll_debug;  // [run histories] or null
    int64_t tally_off;      // batch of h = (h - tally_off) n_batches / n_hist_total
    // eigenvalue generation (sites == null: fixed source, no banking)
    const FissionSite* src; // [run histories] source sites, or null (fixed source)
    double k_norm;          // a collision banks floor(nuSigma_f/Sigma_t/k_norm + xi) sites
    double T_fission;       // Maxwellian temperature of fission neutrons (eV)
    FissionSite* bank;      // staging bank [bank_cap], unordered
    int2* bank_key;         // [bank_cap] {history - first, sequence within the history}
    int64_t bank_cap;
    uint32_t* site_count;   // [run histories] sites each history banked, or null
    EigenCtl* eig;          // or null
};

// Structure-of-arrays particle buffer (one slot per particle in flight) and
// the event queues.
struct Particles {
    int64_t cap = 0;     // slots in use by this run (the particles-in-flight count)
    int64_t stride = 0;  // slots allocated (row stride of W)
    double *x = nullptr, *y = nullptr, *z = nullptr;
    double *u = nullptr, *v = nullptr, *w = nullptr;
    double* E = nullptr;
    double2* sig_ta = nullptr;  // {Sigma_t, Sigma_a} of the last lookup: one 16-byte store and load
    double* sig_nf = nullptr;   // nuSigma_f of the last lookup (eigenvalue runs)
    uint32_t* nsite = nullptr;  // sites banked by the slot's history so far
    double* W = nullptr;  // [MCX_MAX_DMAT][cap] (derivative runs)
    double* cum = nullptr;  // [cap][cum_stride]: running sums C_i of the last lookup, 8 bytes each
                            // (normalised FP32 pairs in the transport's pair form, else FP64)
    int64_t cum_stride = 0; // >= the largest material's species count, a multiple of 4
    int64_t* hist = nullptr;
    uint32_t* rng_n = nullptr;
    uint32_t* ncoll = nullptr;
    int32_t* cell = nullptr;  // ci * n + cj
    int32_t* mat = nullptr;
    int32_t* prob = nullptr;
    uint8_t* flags = nullptr;
    int32_t* q_xs[2] = {nullptr, nullptr};
    int32_t* q_adv[2] = {nullptr, nullptr};
    int32_t* q_dead[2] = {nullptr, nullptr};
    int32_t* q_coll = nullptr;
    int32_t* q_sorted = nullptr;  // binned copy of a queue
    uint32_t* bins = nullptr;     // counting-sort bins
};

// Device-resident loop control: counters, queue sizes, termination.
struct RunCtl {
    unsigned long long next;  // next work item
    long long total;          // work items of the run
    long long iters;
    long long max_iters;
    int n_prob;
    int n_alive;
    int done;
    int error;                // 0 or an MCX_ERR_* code
    int parity;
    int n_xs[2], n_adv[2], n_dead[2];
    int n_coll;
    int sorted;               // this iteration's queue was binned
    int sort_which;           // queue binned this step (fullest mode): 0 XS, 1 collision
    // fullest-queue mode: ring queues (absolute 64-bit positions, modulo the
    // slot count), the ring of the flight queue that receives appends, and
    // the step's selection
    unsigned long long rq_head[5], rq_tail[5];
    int adv_recv;
    int sel;                  // SEL_* of this step, -1 = none
    int sel_ring;             // RQ_* consumed this step
    int pad2;
    unsigned long long sel_begin, sel_end;
    long long sel_count[3];   // steps that ran the lookup / flight / collision kernel
    unsigned long long lk_claim;  // queued mode: next unclaimed entry of the lookup queue
    // queued mode, kernel timing runs: lookups, flights and collisions of the
    // run, and the lookups' running-sum rows (species counts rounded up to 4)
    long long ev_count[4];
};

// Ring queues of the fullest-queue mode and the events that consume them.
enum { RQ_XS = 0, RQ_ADV0 = 1, RQ_ADV1 = 2, RQ_COLL = 3, RQ_DEAD = 4, N_RQ = 5 };
enum { SEL_XS = 0, SEL_ADV = 1, SEL_COLL = 2, SEL_DEAD = 3 };

struct LoopConfig {
    int mode = MCX_QUEUELESS;
    int block = 256;
    int grid = 148;
    int sort_period = 0;
    long long sort_threshold = 20000;
    int n_ebuckets = 128;
    int n_sort_bins = 0;     // materials * n_ebuckets
    float sort_ln_lo = 0.f, sort_scale = 0.f;
    int derivatives = 0;
    int eigen = 0;           // eigenvalue generation: nuSigma_f lookups, fission banking
};

// Kernels of one event-loop iteration, issued on `st` (capturable).
// Returns the number of kernels launched, or -1 on a launch error.
// ev (kernel timing runs, plain launches only): four events recorded around
// the lookup, flight and collision kernels (before the lookup, after each);
// in the queued mode the iteration then also counts the lookups' running-sum
// rows into ctl->ev_count[3] (before the first event).
int launch_iteration(const LoopConfig& c, const Tables& t, const Particles& P,
                     const ProblemDev* probs, const int64_t* work_off, RunCtl* ctl,
                     cudaStream_t st, const cudaEvent_t* ev = nullptr);
// Reset the particle buffer and loop control for a run of `total` work items.
// Fission bank of an eigenvalue generation (eigen.cu): per-history site
// offsets (exclusive scan of the counts; tile_sum needs bank_scan_tiles(n) + 1
// entries, tile_sum[tiles] = total), placement by key, resampling.
int64_t bank_scan_tiles(int64_t n);
int launch_site_offsets(const uint32_t* cnt, int64_t n, unsigned long long* tile_sum,
                        unsigned long long* off, cudaStream_t st);
int launch_bank_order(const FissionSite* bank, const int2* key, int64_t n_banked,
                      const unsigned long long* off, int64_t n_hist, int64_t M, FissionSite* ordered,
                      unsigned long long* bad, int grid, cudaStream_t st);
int launch_bank_resample(const FissionSite* ordered, int64_t M, int64_t N, FissionSite* src, int grid,
                         cudaStream_t st);

int launch_run_init(const LoopConfig& c, const Particles& P, RunCtl* ctl, long long total,
                    int n_prob, long long max_iters, cudaStream_t st);

}  // namespace mcx
