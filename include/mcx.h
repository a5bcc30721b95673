/*
 * mcx.h -- C ABI of libmcx: event-based Monte Carlo particle transport and the
 * macroscopic cross-section lookup on one NVIDIA B300 (sm_103a).
 *
 * Paper: "Integrating ytopt and libEnsemble to Autotune OpenMC" (arXiv
 * 2402.09222).  Sec. 5.1 describes what is computed here: OpenMC's
 * event-based mode, a buffer of particles in flight refilled after each
 * kernel call, the macroscopic cross-section lookup ("the most expensive
 * kernel": a search of every species' energy grid, narrowed by a logarithmic
 * hash grid), queued or queueless event logic, and sorting by material and
 * energy above a minimum queue size.  Table 1 lists the tunable parameters.
 *
 * Conventions (all entry points):
 *   - every call returns an int status (MCX_OK or a negative MCX_ERR_*);
 *     nothing aborts or throws across the ABI; mcx_last_error() returns a
 *     thread-local message for the last failing call on the calling thread;
 *   - input arrays passed as host pointers are copied; the caller keeps
 *     ownership and may free them when the call returns;
 *   - arguments documented as DEVICE pointers must be device memory on the
 *     problem's device (e.g. from torch.empty(..., device="cuda")); they are
 *     borrowed until the asynchronous work queued on `stream` completes;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream);
 *   - an mcx_problem is not thread-safe: one thread at a time per handle.
 */
#ifndef MCX_H
#define MCX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define MCX_OK 0
#define MCX_ERR_ARG (-1)        /* invalid argument (message says which) */
#define MCX_ERR_CUDA (-2)       /* a CUDA runtime call failed */
#define MCX_ERR_OOM (-3)        /* device or host allocation failed */
#define MCX_ERR_ITER_LIMIT (-4) /* the event loop reached its iteration cap */
#define MCX_ERR_STATE (-5)      /* call out of order (e.g. run before tables) */
#define MCX_ERR_BOUNDS (-6)     /* a device-side bounds check fired */
#define MCX_ERR_TIMEOUT (-7)    /* the run exceeded its host time limit */

/* ---- enumerations ---------------------------------------------------- */
/* Geometry of a problem.  NONE: a handle that only holds cross-section
 * tables (for the lookup entry points). */
#define MCX_GEOM_INFINITE 0 /* one material everywhere, source at origin */
#define MCX_GEOM_LATTICE 1  /* n x n pin lattice in a box, see below */
#define MCX_GEOM_SLAB 2     /* x in [0, L], pencil beam along +x */
#define MCX_GEOM_NONE 3

/* Storage precision of the sigma tables (energies are always FP64). */
#define MCX_FP64 0
#define MCX_FP32 1

/* Event logic (Sec. 5.1, "queuing logic"). */
#define MCX_QUEUELESS 0       /* every event kernel visits every slot */
#define MCX_QUEUED 1          /* every event kernel runs each iteration over its
                                 device-built compacted queue (the flight,
                                 whose queue holds every live particle, over
                                 the slots while at least three quarters of
                                 them are live) */
#define MCX_QUEUED_FULLEST 2  /* the paper's queued policy, decided on the device:
                                 each step runs only the event kernel whose
                                 queue (needs lookup / flight / collision /
                                 refill) holds the most particles */

/* Lookup options for mcx_xs_lookup (bit flags). */
#define MCX_LOOKUP_EXACT 0 /* FP64 arithmetic, bit-identical to the plain definition */
#define MCX_LOOKUP_FAST 1  /* FP32 interpolation weights, compensated sums (<= 1e-6 rel) */
#define MCX_LOOKUP_SORT 2  /* bin lookups by (material, log-energy) before the gather */
#define MCX_LOOKUP_STAGED 4 /* with FAST and a binned order: stage each chunk's grid
                               points in shared memory by TMA bulk copies (same
                               results, bit for bit) */
#define MCX_LOOKUP_OUT32 8  /* with FAST: out holds FP32 values (the compensated
                               sum rounded once; still within 1e-6 relative),
                               half the output bytes */
#define MCX_LOOKUP_LINEAR 16 /* with FAST and a binned order: per 64-lookup
                               round, the species whose grid interval holds
                               every lookup of the round (or whose grid has one
                               point inside the round's energy range) are summed
                               once per round as one linear function of E (plus
                               a hinge at that point), the rest per lookup.
                               Within the same 1e-6 relative bound as FAST, but
                               not bit-identical to it, and the last bits depend
                               on which lookups share a round.  Ignored with
                               STAGED. */
#define MCX_LOOKUP_BINNED_INPUTS 32 /* mcx_xs_lookup_ordered only: E and mat
                               are already in the processing order (see there) */

/* Problem flags. */
#define MCX_FLAG_DERIVATIVES 1   /* likelihood-ratio density-derivative tallies */
#define MCX_FLAG_HISTORY_DEBUG 2 /* keep per-history collision counts */

/* Tallies (mcx_read_tallies `which`).  Shapes, with B batches, nb bins
 * (energy bins for INFINITE, regions for LATTICE, 1 for SLAB) and M
 * materials:  FLUX, ABSORB [B][nb];  OUTCOME [B][5] = {absorbed, leaked
 * through the +x face, leaked elsewhere, cut off, collisions};  DFLUX,
 * DABSORB [B][nb][M];  DOUTCOME [B][5][M]. */
#define MCX_TALLY_FLUX 0
#define MCX_TALLY_ABSORB 1
#define MCX_TALLY_OUTCOME 2
#define MCX_TALLY_DFLUX 3
#define MCX_TALLY_DABSORB 4
#define MCX_TALLY_DOUTCOME 5

#define MCX_MAX_DMAT 4 /* materials supported by the derivative tallies */

typedef struct mcx_problem mcx_problem; /* opaque, owned by the library */

/* Problem description.  All pointers are HOST pointers and are copied.
 *
 * LATTICE (the 17x17 pin-cell workload of the paper's benchmark class): pins
 * of radius `radius` on a square lattice of `lattice_n`^2 cells of side
 * `pitch`, centred on the origin; the box's x/y faces are vacuum, the planes
 * z = 0 and z = height are reflective.  Regions: pin (i, j) = i * n + j,
 * moderator = n^2; `region_material` has n^2 + 1 entries.  Each history
 * starts at the centre of a uniformly chosen pin at z = height / 2.
 * INFINITE: `region_material` has 1 entry; tallies bin by energy with the
 * `n_ebins` + 1 increasing edges.  SLAB: 1 region, tally bin 0.
 * All histories start with energy E0, isotropic (LATTICE, INFINITE) or along
 * +x (SLAB), and die when a scattering leaves them below E_cut.
 * History h belongs to batch floor(h * n_batches / n_histories). */
typedef struct {
    int32_t geometry;
    int32_t lattice_n;
    double pitch, radius, height, slab_length;
    int32_t n_regions;
    const int32_t* region_material;
    double E0, E_cut;
    int32_t n_ebins;
    const double* ebin_edges;
    int32_t n_batches;
    uint32_t problem_id; /* part of the random-number key */
    int64_t n_histories; /* total histories of the problem (defines batches) */
    int32_t flags;       /* MCX_FLAG_* */
    int32_t device;      /* CUDA device ordinal */
} mcx_problem_desc;

/* Event-loop tuning (Table 1 of the paper, mapped to this GPU).
 *   mode            MCX_QUEUELESS, MCX_QUEUED or MCX_QUEUED_FULLEST
 *   block_size      threads per block of the event kernels (32..1024, /32)
 *   sort_period     bin the lookup queue (queued mode) or the selected
 *                   lookup or collision segment (fullest queue) every this
 *                   many iterations (0 = never); queued modes only
 *   sort_threshold  ...and only when a queue holds at least this many
 *                   particles (the paper's minimum sorting threshold)
 *   iters_per_sync  event-loop iterations captured per CUDA graph launch
 *                   between host checks of the termination flag (>= 1)
 *                   (in MCX_QUEUED_FULLEST an iteration is one step: a
 *                   refill and the one event kernel selected)
 *   max_event_iters iteration cap of one run (0 = automatic); reaching it
 *                   returns MCX_ERR_ITER_LIMIT instead of looping on
 *   use_graph       1 = replay the captured loop body, 0 = plain launches
 *   time_limit_s    wall-clock budget of one run in seconds (0 = none),
 *                   checked by the host between graph launches; when it is
 *                   exceeded the run stops after the iterations in flight and
 *                   returns MCX_ERR_TIMEOUT (tallies then hold a partial run).
 *                   Used by the autotuner for the paper's evaluation time
 *                   limit (1.5 x the baseline run time). */
typedef struct {
    int32_t mode;
    int32_t block_size;
    int32_t sort_period;
    int64_t sort_threshold;
    int32_t iters_per_sync;
    int64_t max_event_iters;
    int32_t use_graph;
    double time_limit_s;
} mcx_tune;

/* Create a problem on desc->device.  Validates the description (geometry
 * sizes, region materials in range once tables are loaded, batches >= 1,
 * n_histories >= 1, increasing energy-bin edges).  *out receives the handle.
 * Errors: MCX_ERR_ARG, MCX_ERR_CUDA, MCX_ERR_OOM. */
int mcx_init_problem(const mcx_problem_desc* desc, mcx_problem** out);

/* Load the species library and materials (Sec. 5.1: per-species energy grids
 * and reaction cross sections; materials as lists of species with atom
 * densities).  HOST pointers, copied:
 *   grid_offsets [n_species+1]  species s owns points [off[s], off[s+1]),
 *                               at least 2 per species
 *   energies     [P]            FP64, positive, finite, strictly increasing
 *                               within each species
 *   sigma        [P][n_ch]      FP64 cross sections, finite and >= 0;
 *                               n_ch = 2 (scatter, absorb), 3 (scatter,
 *                               absorb, nu-fission) or 5 (total, scatter,
 *                               absorb, fission, nu-fission); the lookup
 *                               entry points take any n_ch in 1..5
 *   awr          [n_species]    mass ratio A >= 1 (used by transport)
 *   mat_offsets  [n_materials+1], mat_species [nnz] (ids in range),
 *   mat_dens     [nnz]          atom densities, finite and >= 0
 *   precision    MCX_FP64 or MCX_FP32 (sigma is rounded to FP32 on upload)
 *   hash_bins    number of logarithmic hash-grid bins over [min, max] of all
 *                grids (0 = no hash: full binary searches); Table 1 range
 *                100..100000, default 4000
 * Replaces previously loaded tables.  Errors: MCX_ERR_ARG (with the first
 * offending index in the message), MCX_ERR_OOM, MCX_ERR_CUDA. */
int mcx_load_xs_tables(mcx_problem* p, int32_t n_species, const int64_t* grid_offsets,
                       const double* energies, const double* sigma, int32_t n_ch,
                       const double* awr, int32_t n_materials, const int32_t* mat_offsets,
                       const int32_t* mat_species, const double* mat_dens, int32_t precision,
                       int32_t hash_bins);

/* Make `dst` use the tables and materials already loaded into `src` (no
 * copy; `src` must outlive `dst`'s use of them).  Used for many problems over
 * one library.  Errors: MCX_ERR_ARG, MCX_ERR_STATE (src has no tables). */
int mcx_share_xs_tables(mcx_problem* dst, const mcx_problem* src);

/* Rebuild the hash grid with a new bin count (0 = none) without reloading
 * the tables.  Results of every entry point are independent of it. */
int mcx_set_hash_bins(mcx_problem* p, int32_t hash_bins);

/* Replace the atom densities (same sparsity as loaded), HOST pointer. */
int mcx_set_densities(mcx_problem* p, const double* mat_dens, int64_t nnz);

/* Replace densities and/or cross sections from DEVICE buffers (same shapes
 * as loaded: mat_dens [nnz] FP64, sigma [P][n_ch] FP64; either may be NULL to
 * keep the current values), queued on `stream`.  FP32 tables receive the
 * values rounded to FP32.  No validation of the values is done on this path
 * (it serves gradient checks and optimisation loops that own the buffers).
 * Errors: MCX_ERR_ARG, MCX_ERR_STATE, MCX_ERR_CUDA. */
int mcx_update_tables_device(mcx_problem* p, const double* mat_dens, const double* sigma,
                             void* stream);

/* Set / get the event-loop tuning.  mcx_default_tuning fills the plain form:
 * queueless, block 256, no sorting, threshold 20000, 16 iterations per sync,
 * automatic cap, graphs on. */
void mcx_default_tuning(mcx_tune* t);
int mcx_set_tuning(mcx_problem* p, const mcx_tune* t);

/* Run histories [first_history, first_history + n_histories) of the problem
 * with a buffer of `particles_in_flight` slots (Sec. 5.1: dead slots are
 * refilled from the remaining histories after every event iteration; the
 * count does not change any history).  Scores add to the problem's tallies.
 * Random numbers: Philox4x32-10 keyed by (seed, problem_id), one stream per
 * history, so results do not depend on the slot count, tuning or order.
 * Queued on `stream`; returns after the last iteration has been issued and
 * the termination flag read (the host synchronises with `stream` once per
 * `iters_per_sync` iterations).  Errors: MCX_ERR_ARG, MCX_ERR_STATE (no
 * tables), MCX_ERR_ITER_LIMIT, MCX_ERR_BOUNDS, MCX_ERR_CUDA, MCX_ERR_OOM. */
int mcx_run_batch(mcx_problem* p, int64_t first_history, int64_t n_histories,
                  int64_t particles_in_flight, uint64_t seed, void* stream);

/* Many independent problems in one persistent event loop (one slot buffer,
 * one CUDA graph): histories of all problems are drawn from one global work
 * list.  All problems must share one set of tables (mcx_share_xs_tables) and
 * have the derivative flag off.  Each problem's histories [0, n_hist[i]) are
 * run and scored into that problem's own tallies; problems[0]'s tuning is
 * used.  Errors as mcx_run_batch. */
int mcx_batch_run(int32_t n_problems, mcx_problem* const* problems, const int64_t* n_hist,
                  int64_t particles_in_flight, uint64_t seed, void* stream);

/* k-eigenvalue power iteration (the paper's benchmark, Hoogenboom-Martin, is a
 * criticality problem, Sec. 5.1).  Generation g runs n_per_gen histories with
 * ids g * n_per_gen + i (their own random streams) through the event loop
 * under the problem's tuning.  Generation 0 starts from the fixed source of
 * the description; generation g > 0 starts history i at site i of its
 * source: isotropic, with an energy from the Maxwellian fission spectrum of
 * temperature T_fission (eV).  Every collision, before its reaction is
 * decided, banks floor(nuSigma_f / Sigma_t / k_norm + xi) sites at the
 * collision point (xi: the collision's fourth uniform); k_norm = k0 in
 * generation 0 and the previous generation's k afterwards.  The M banked
 * sites are put in the order of their parent history and, within a history,
 * of banking; the next source is source[i] = bank[floor(i M / n_per_gen)].
 * Per generation, HOST gen_out[4 g .. 4 g + 3] = {k = M k_norm / n_per_gen,
 * collision estimate sum(nuSigma_f / Sigma_t) / n_per_gen, track-length
 * estimate sum(d nuSigma_f) / n_per_gen, M}.  The tallies are cleared at the
 * first active generation and then score the last n_generations - n_inactive
 * generations: active history j = (g - n_inactive) n_per_gen + i falls in
 * batch floor(j n_batches / ((n_generations - n_inactive) n_per_gen)).  The
 * bank holds 4 n_per_gen sites (at least 4096) and grows when an inactive
 * generation overflows it (the generation is run again).  Needs 3-channel
 * (scatter, absorb, nu-fission) or 5-channel tables and no derivative flag.
 * Synchronous.  Errors: MCX_ERR_ARG, MCX_ERR_STATE (a generation banked no
 * site, or an inconsistent bank), MCX_ERR_BOUNDS (an active generation
 * overflowed the bank), MCX_ERR_ITER_LIMIT, MCX_ERR_TIMEOUT, MCX_ERR_CUDA,
 * MCX_ERR_OOM. */
int mcx_run_eigenvalue(mcx_problem* p, int64_t n_per_gen, int32_t n_generations, int32_t n_inactive,
                       double k0, double T_fission, int64_t particles_in_flight, uint64_t seed,
                       double* gen_out, void* stream);

/* Waits for `stream` and reports whether a staged lookup (MCX_LOOKUP_STAGED)
 * on this handle gave up on its shared-memory pipeline since the last check
 * (a bounded wait ran out; never expected): MCX_ERR_TIMEOUT, and the flag is
 * cleared; MCX_OK otherwise.  In the bounds-checked build (libmcx_bounds.so,
 * mcx_bounds_checked() == 1) it first reports the first index check that
 * failed on the handle's device since the last check, in any kernel:
 * MCX_ERR_BOUNDS with the site and index in mcx_last_error (the check
 * skipped or clamped the access; the outputs of the lookups involved are
 * left unwritten), and the record is cleared.  Host-synchronous. */
int mcx_check_device(mcx_problem* p, void* stream);

/* 1 in the bounds-checked build of the library (compiled with
 * MCX_BOUNDS_CHECK=1: the kernels check processing-order indices, hash-grid
 * windows, event-queue slots and appends, tally bins and collision
 * materials before using them, and report failures as MCX_ERR_BOUNDS from
 * mcx_check_device and the transport runs), 0 in the release build. */
int mcx_bounds_checked(void);

/* The last eigenvalue generation's ordered bank: its size, and its first n
 * sites as HOST rows {x, y, z, ci, cj, inpin} (n <= size).  Synchronous. */
int mcx_fission_bank_size(const mcx_problem* p, int64_t* n);
int mcx_read_fission_bank(mcx_problem* p, double* rows, int64_t n);

/* Size in doubles of a tally, and a synchronous copy of it to HOST memory
 * (n must equal the size).  mcx_zero_tallies clears all tallies. */
int mcx_tally_size(const mcx_problem* p, int32_t which, int64_t* n);
int mcx_read_tallies(mcx_problem* p, int32_t which, double* host_out, int64_t n);
int mcx_zero_tallies(mcx_problem* p);

/* Per-history collision counts of the last mcx_run_batch (requires
 * MCX_FLAG_HISTORY_DEBUG): ncoll[i] for history first_history + i, HOST
 * pointer, n <= that run's n_histories.  Synchronous. */
int mcx_read_history_debug(mcx_problem* p, uint32_t* ncoll, int64_t n);

/* Kernel timing (an instrument of this library, no counterpart in the
 * paper): with on = 1, later runs of the handle launch their event loop
 * without graph capture and record CUDA events around the lookup, flight and
 * collision kernels of every iteration (a run is slower than with graphs; its
 * results are the same).  Errors: MCX_ERR_ARG. */
int mcx_set_kernel_timing(mcx_problem* p, int32_t on);

/* After a run with kernel timing on: ms[3] = summed device time of the
 * lookup, flight and collision kernels (-1 when timing was off); counts[4] =
 * lookups, flights and collisions of the run and the summed lengths of the
 * running-sum rows the lookups wrote (each material's species count rounded
 * up to a multiple of 4), in the queued mode (MCX_QUEUED); -1 in the other
 * modes.  The counts are kept for every run.  Errors: MCX_ERR_ARG. */
int mcx_last_kernel_stats(const mcx_problem* p, double* ms, int64_t* counts);

/* Event-loop statistics of the last run: out[0] iterations (steps in
 * MCX_QUEUED_FULLEST), out[1] graph launches, out[2] kernel launches, and
 * when n >= 6, out[3..5] the steps that selected the lookup, flight and
 * collision queue (MCX_QUEUED_FULLEST; 0 otherwise).  HOST pointer, n >= 3.
 * An inconsistent queue state found on the device ends a run with
 * MCX_ERR_STATE. */
int mcx_last_run_stats(const mcx_problem* p, int64_t* out, int32_t n);

/* Macroscopic cross-section lookup (Sec. 5.1, "the most expensive kernel"):
 *   out[l][r] = sum over the species i of material mat[l] of
 *               N_i * sigma_{r,i}(E[l]),  r = 0..n_ch-1,
 * where sigma_{r,i} interpolates species i's table linearly in energy on the
 * grid interval [g[k], g[k+1]] with k the largest index in [0, n-2] such
 * that g[k] <= E (k = 0 below the grid, n-2 at or above its top; the
 * fraction is clamped to [0, 1]).  E (FP64 [n]), mat (int32 [n]) and out
 * (FP64 [n][n_ch], row-major; FP32 with MCX_LOOKUP_OUT32) are DEVICE
 * pointers.  flags: MCX_LOOKUP_EXACT
 * gives the plain definition's FP64 result bit for bit (species in stored
 * order, sums from +0.0, no fused multiply-add); MCX_LOOKUP_FAST stays within
 * 1e-6 relative of it; MCX_LOOKUP_SORT first bins the lookups by material and
 * log-energy (results unchanged; uses library-owned scratch memory sized for
 * n; with MCX_LOOKUP_FAST from 2^22 lookups the binning also hands the
 * energies and materials over in the binned order, as mcx_xs_sort_inputs,
 * 12 more bytes per lookup of scratch); MCX_LOOKUP_LINEAR with FAST and SORT sums per 64-lookup round where it
 * can (within the same bound, last bits depending on the order within a
 * bin); MCX_LOOKUP_OUT32 writes FP32 outputs.  A material id out of range
 * gives NaN outputs for that lookup.
 * Errors: MCX_ERR_ARG, MCX_ERR_STATE, MCX_ERR_CUDA, MCX_ERR_OOM. */
int mcx_xs_lookup(mcx_problem* p, int64_t n, const double* E, const int32_t* mat, void* out,
                  int32_t flags, void* stream);

/* Binning of lookups by material and energy (Sec. 5.1: sorting so that
 * neighbouring threads work on the same material and nearby energies):
 * perm (int32 [n], DEVICE) receives 0..n-1 ordered by (material, bucket of
 * log E) with max(n / (materials x 128), 16384) equal buckets per material
 * over the library's energy range (fewer when materials x buckets would
 * exceed 2^21 bins; at least 1), so about 128 lookups per bucket in large
 * batches.  Order within a bucket is unspecified.  E and mat are
 * DEVICE pointers.  Batches of 2^22 lookups and more are binned in two
 * levels (counts per tile and coarse bin in shared memory, then each coarse
 * bin ranked by its fine bins in shared memory), smaller ones by a counting
 * sort with global counters.  Uses library-owned scratch, allocated on first
 * use and kept with the handle: the bin counters, and for two-level batches
 * 10 bytes per lookup.  Errors: MCX_ERR_ARG, MCX_ERR_STATE, MCX_ERR_CUDA,
 * MCX_ERR_OOM. */
int mcx_xs_sort(mcx_problem* p, int64_t n, const double* E, const int32_t* mat, int32_t* perm,
                void* stream);

/* mcx_xs_sort that also hands over the inputs in the binned order:
 * E_binned[j] = E[perm[j]] and mat_binned[j] = mat[perm[j]], or -1 where
 * that material id is outside [0, n_materials) (FP64 [n] and int32 [n],
 * DEVICE, caller-owned, not aliasing E or mat), for mcx_xs_lookup_ordered
 * with MCX_LOOKUP_BINNED_INPUTS, which then reads them in sequence instead
 * of through the permutation.  Two-level batches carry each energy with its
 * index through both binning passes (8 more bytes per lookup of
 * library-owned scratch, 18 in all) and take the material from its bin;
 * smaller batches gather them after the sort.  Errors as mcx_xs_sort. */
int mcx_xs_sort_inputs(mcx_problem* p, int64_t n, const double* E, const int32_t* mat, int32_t* perm,
                       double* E_binned, int32_t* mat_binned, void* stream);

/* mcx_xs_lookup processing the lookups in the order perm (a permutation of
 * 0..n-1, e.g. from mcx_xs_sort; NULL = natural order).  Results land in each
 * lookup's own row of out, so the order changes no value (with
 * MCX_LOOKUP_LINEAR: within its bound).  flags may hold MCX_LOOKUP_FAST,
 * MCX_LOOKUP_STAGED (applies to a binned perm with MCX_LOOKUP_FAST;
 * mcx_check_device reports a pipeline that gave up), MCX_LOOKUP_OUT32,
 * MCX_LOOKUP_LINEAR and MCX_LOOKUP_BINNED_INPUTS (with MCX_LOOKUP_FAST and a
 * perm, not with MCX_LOOKUP_STAGED: E and mat are given in the processing
 * order, lookup j taking E[j] and mat[j] and writing row perm[j] of out, as
 * mcx_xs_sort_inputs produces them; the results equal those from the
 * original E and mat bit for bit).  DEVICE pointers. */
int mcx_xs_lookup_ordered(mcx_problem* p, int64_t n, const double* E, const int32_t* mat,
                          const int32_t* perm, void* out, int32_t flags, void* stream);

/* The binned lookup (mcx_xs_lookup with MCX_LOOKUP_SORT) for callers that
 * cannot allocate device memory -- for example a process whose device memory
 * is reserved up front by another allocator, or a latency-bound loop that
 * cannot afford cudaMalloc's implicit synchronisation.  The paper has no
 * counterpart; this is an interface convenience of the library.
 * Its scratch (binning permutation and bin counters) lives in fixed-size
 * device arrays of the library, about 4.05 MB per device, created when the
 * library is loaded onto a device and kept until the process exits; the call
 * itself allocates nothing.  Inputs and outputs are the caller's DEVICE
 * buffers, as for mcx_xs_lookup; flags may hold MCX_LOOKUP_FAST.
 * Limits: n <= MCX_STATIC_MAX_LOOKUPS; the binning uses at most
 * MCX_STATIC_MAX_BINS bins (energy buckets per material are reduced to fit),
 * and more materials than that fail with MCX_ERR_ARG.
 * The first call on a device looks up the scratch's device address (a
 * one-time set-up per device) and keeps it for the life of the process;
 * make that first call before any stream capture, and do not use the entry
 * point on a device after cudaDeviceReset (or any other teardown of its
 * primary context) in the same process: the scratch may then live at
 * another address.  All calls on a device share the one scratch: calls that overlap
 * on the GPU (e.g. on two streams at once) race and give wrong results; order
 * them on one stream or with events.
 * Errors: MCX_ERR_ARG, MCX_ERR_STATE, MCX_ERR_CUDA. */
#define MCX_STATIC_MAX_LOOKUPS 1048576
#define MCX_STATIC_MAX_BINS 12288
int mcx_xs_lookup_binned_static(mcx_problem* p, int64_t n, const double* E, const int32_t* mat,
                                double* out, int32_t flags, void* stream);

/* The same lookup from HOST buffers: copies in, computes and copies out in
 * chunks of up to 2M lookups (4M with MCX_LOOKUP_OUT32) pipelined over three
 * streams (with MCX_LOOKUP_SORT each chunk is binned on the device);
 * synchronous.  Device staging of about 3 x chunk x (32 + 8 n_ch) bytes is
 * allocated on first use and kept with the handle.  out_host is FP64
 * [n][n_ch], or FP32 with MCX_LOOKUP_OUT32 (half the device-to-host bytes,
 * which bound this path).  Host buffers should be pinned (cudaHostAlloc /
 * torch pin_memory) for full copy speed. */
int mcx_xs_lookup_host(mcx_problem* p, int64_t n, const double* E_host, const int32_t* mat_host,
                       void* out_host, int32_t flags);

/* Grid indices used by the lookup, for parity tests: kout[l * max_species +
 * i] = k of the i-th species of material mat[l], -1 past its species count.
 * DEVICE pointers.  max_species must be >= the largest material. */
int mcx_xs_indices(mcx_problem* p, int64_t n, const double* E, const int32_t* mat,
                   int32_t max_species, int32_t* kout, void* stream);

/* Adjoint of mcx_xs_lookup (exact arithmetic) for a cotangent grad_out
 * [n][n_ch]:
 *   grad_dens[j]             += sum_l sum_r grad_out[l][r] * sigma_{r,s}(E_l)
 *   grad_sigma[p_k][r]       += N_j (1 - f) grad_out[l][r]
 *   grad_sigma[p_{k+1}][r]   += N_j f grad_out[l][r]
 * for every lookup l whose material holds entry j (species s, density N_j).
 * grad_dens [nnz] and grad_sigma [P][n_ch] are FP64 DEVICE buffers that are
 * accumulated into (zero them first).  E, mat, grad_out are DEVICE pointers.
 * The lookups are binned first (material, log-energy bucket; finer than
 * mcx_xs_sort's, about 8 lookups per bucket) into the handle's scratch,
 * allocated on first use as for MCX_LOOKUP_SORT; warps of
 * one material then sum their contributions per species and grid interval
 * (exact FP64 fractions, sums over energy-sorted lanes) before one atomic
 * per point and channel, and the density gradients per block before one
 * atomic per entry.  Summation order is not fixed (atomics), so results match
 * a sequential sum to rounding (within 1e-11 relative in the tests).  Lookups
 * with an out-of-range material or a NaN energy contribute nothing; calls on
 * one handle share its scratch and are ordered on one stream. */
int mcx_xs_lookup_backward(mcx_problem* p, int64_t n, const double* E, const int32_t* mat,
                           const double* grad_out, double* grad_dens, double* grad_sigma,
                           void* stream);

/* Test hook: n Philox4x32-10 uniforms of one history stream, as the
 * transport kernels draw them (uniform first+i of history `hist`), into a
 * DEVICE buffer out [n]. */
int mcx_debug_uniforms(uint64_t seed, uint32_t problem_id, uint64_t hist, uint32_t first,
                       int64_t n, double* out, void* stream);

/* Test hook: the flight length -ln x as the transport computes it (a
 * table-driven logarithm, Tang 1990) and as the CUDA library computes it,
 * for n values x in [2^-53, 1) (the range of the uniforms; others are out of
 * its domain) in a DEVICE buffer; out [n][2] (DEVICE) receives the pairs. */
int mcx_debug_neg_log(const double* x, int64_t n, double* out, void* stream);

/* Test hook: the transport's macroscopic lookup (FP32-pair sums from the
 * stored per-point slopes and totals) for n lookups (energies E, materials
 * mat; DEVICE buffers): out [n][3] (DEVICE) receives Sigma_t, Sigma_a and
 * nuSigma_f (0 without a nu-fission channel), NaN for an out-of-range
 * material or a NaN energy.  Synchronises `stream`; allocates a scratch of
 * n times the largest material's species count of 8-byte sums.  n <= 2^24;
 * the tables must have 2, 3 or 5 channels, as for transport.
 * Errors: MCX_ERR_STATE (no tables), MCX_ERR_ARG, MCX_ERR_OOM, MCX_ERR_CUDA. */
int mcx_debug_transport_xs(mcx_problem* p, int64_t n, const double* E, const int32_t* mat, double* out,
                           void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* mcx_last_error(void);

/* Library version string. */
const char* mcx_version(void);

/* Release the problem and all device memory it owns.  NULL is ignored. */
void mcx_destroy(mcx_problem* p);

#ifdef __cplusplus
}
#endif
#endif /* MCX_H */
