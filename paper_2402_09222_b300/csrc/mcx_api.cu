// mcx_api.cu -- the C ABI of libmcx (declared in include/mcx.h): argument
// validation, device memory, the event-loop driver (CUDA-graph replay with a
// device-side termination flag and iteration cap) and the lookup entry
// points.  No exception or abort crosses the ABI: every failure becomes a
// status code plus a thread-local message.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <chrono>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.h"

using namespace mcx;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

// MCX_ERR_BOUNDS with the site and index of a bounds-checked build's error
// word (site << 56 | index).
int bounds_failure(unsigned long long word, const char* unit)
{
    static const char* const site[] = {"?", "lookup index from the processing order",
                                       "hash-grid search window", "particle slot from an event queue",
                                       "event-queue append", "tally bin", "collision material"};
    const int k = (int)(word >> 56);
    const long long idx = (long long)(word & ((1ull << 56) - 1ull));
    return fail(MCX_ERR_BOUNDS, "%s: %s out of bounds (index %lld)", unit, site[k >= 1 && k <= 6 ? k : 0], idx);
}

#define CUDA_TRY(expr)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (expr);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            if (e_ == cudaErrorMemoryAllocation) {                                        \
                cudaGetLastError();                                                       \
                return fail(MCX_ERR_OOM, "%s: %s", #expr, cudaGetErrorString(e_));        \
            }                                                                             \
            return fail(MCX_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_));           \
        }                                                                                 \
    } while (0)

#define TRY(expr)                  \
    do {                           \
        int r_ = (expr);           \
        if (r_ != MCX_OK) return r_; \
    } while (0)

// Selects a device for the duration of a call and restores the caller's.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Fault injection on the host: with MCX_FAIL_ALLOC_AFTER=N in the
// environment, the device allocations after the first N (counted while the
// variable is set) fail with MCX_ERR_OOM without reaching the driver.
bool simulated_alloc_failure()
{
    static std::atomic<long long> count{0};
    const char* v = std::getenv("MCX_FAIL_ALLOC_AFTER");
    if (!v || !*v) {
        count.store(0);
        return false;
    }
    return count.fetch_add(1) + 1 > std::atoll(v);
}

template <typename T>
int dev_alloc(T** p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    if (simulated_alloc_failure())
        return fail(MCX_ERR_OOM, "cudaMalloc(%zu bytes): simulated failure (MCX_FAIL_ALLOC_AFTER)",
                    sizeof(T) * count);
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? MCX_ERR_OOM : MCX_ERR_CUDA,
                    "cudaMalloc(%zu bytes): %s", sizeof(T) * count, cudaGetErrorString(e));
    }
    return MCX_OK;
}

template <typename T>
void dev_free(T*& p)
{
    if (p) cudaFree((void*)p);
    p = nullptr;
}

// Tables and materials on the device, shared by reference count.
struct TableStore {
    int refs = 1;
    int device = 0;
    Tables view;
    int64_t* goff = nullptr;
    double* E = nullptr;
    double* winv = nullptr;   // per interval 1 / (g[k+1] - g[k]) (transport)
    double* slope = nullptr;  // per interval and channel, from the device sigma table (transport)
    double2* ttot = nullptr;  // per point total of scatter and absorption and its slope (transport)
    float4* tpair = nullptr;  // the transport's values as FP32 pairs
    float2* mden2 = nullptr;  // densities as FP32 pairs
    float4* frec = nullptr;
    void* sigma = nullptr;
    double* awr = nullptr;
    double* inv_a1sq = nullptr;   // per species 1 / (A + 1)^2
    int32_t* moff = nullptr;
    int32_t* msp = nullptr;
    double* mden = nullptr;
    int4* ment = nullptr;
    std::vector<int4> h_ment;
    bool h_ment_stale = false;  // densities were last set from device buffers
    int32_t max_points = 0;
    int32_t* hidx = nullptr;
    double* hbound = nullptr;
    double emin = 0.0, emax = 0.0;
    int64_t nnz = 0;
    std::vector<int32_t> h_moff;

    ~TableStore()
    {
        dev_free(goff);
        dev_free(E);
        dev_free(winv);
        dev_free(slope);
        dev_free(ttot);
        dev_free(tpair);
        dev_free(mden2);
        dev_free(frec);
        if (sigma) cudaFree(sigma);
        dev_free(awr);
        dev_free(inv_a1sq);
        dev_free(moff);
        dev_free(msp);
        dev_free(mden);
        dev_free(ment);
        dev_free(hidx);
        dev_free(hbound);
    }
};

int sm_count_of(int device)
{
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n <= 0)
        n = 148;
    return n;
}

}  // namespace

// Host-path pipeline of mcx_xs_lookup_host: chunks of kHostChunk lookups go
// round-robin over kHostSlots streams, each with its own staging and binning
// scratch (copy in, bin, look up, copy out), so the device-to-host copies of
// one chunk overlap the copy-in and compute of the next ones.  1e8 lookups
// on 3 streams: FP64 outputs (5.2 GB over the host link, which bounds them)
// 73.6 ms in 2M-lookup chunks, 74.6 in 4M; FP32 outputs (3.2 GB; the
// per-chunk lookups weigh more) 43.2 ms in 4M chunks, 48.5 in 2M.
#ifndef MCX_HOST_SLOTS
#define MCX_HOST_SLOTS 3
#endif
#ifndef MCX_HOST_CHUNK
#define MCX_HOST_CHUNK (2 << 20)
#endif
#ifndef MCX_HOST_CHUNK32
#define MCX_HOST_CHUNK32 (4 << 20)
#endif
constexpr int kHostSlots = MCX_HOST_SLOTS;
constexpr int64_t kHostChunk = MCX_HOST_CHUNK;
constexpr int64_t kHostChunk32 = MCX_HOST_CHUNK32;
static_assert(kHostSlots >= 1 && kHostSlots <= 4, "host pipeline slots: 1 to 4 streams");
constexpr int kWorkCtrs = 4;   // chunk counters (>= kHostSlots), then the error word

struct mcx_problem {
    mcx_problem_desc desc{};
    std::vector<int32_t> region_material;
    std::vector<double> ebin_edges;
    int device = 0;
    int sm_count = 148;
    int nb = 0;  // tally bins
    int M = 0;   // derivative materials (0 = off)
    TableStore* tables = nullptr;
    mcx_tune tune{};
    // device copies of the description
    int32_t* d_region_material = nullptr;
    double* d_lattice = nullptr;   // lattice plane and centre coordinates (2 n + 1)
    double* d_ebin_edges = nullptr;
    // tallies
    double* flux = nullptr;
    double* absorb = nullptr;
    double* outcome = nullptr;
    double* dflux = nullptr;
    double* dabsorb = nullptr;
    double* doutcome = nullptr;
    // run resources
    Particles P;
    void* p_block = nullptr;
    int64_t p_cap = 0;
    bool p_has_w = false;
    size_t bins_cap = 0;
    ProblemDev* d_probs = nullptr;
    int64_t* d_work_off = nullptr;
    int probs_cap = 0;
    RunCtl* d_ctl = nullptr;
    RunCtl* h_ctl = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t stream2 = nullptr;
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<unsigned char> graph_key;
    uint32_t* ncoll_debug = nullptr;
    int64_t debug_cap = 0;
    int64_t debug_n = 0;
    // lookup scratch
    int32_t* perm = nullptr;
    uint32_t* lbins = nullptr;
    int32_t* bin2 = nullptr;   // two-level binning: bin keys [n], lookup indices [n], fine bins [n] uint16
    double* bin_E = nullptr;   // energies and materials handed over in the binned order [n]
    int32_t* bin_M = nullptr;
    int64_t perm_cap = 0;
    int64_t bin_in_cap = 0;
    size_t lbins_cap = 0;
    size_t bin2_cap = 0;
    double* h_buf = nullptr;  // host-path device staging
    unsigned long long* work_ctr = nullptr;  // chunk counters of the binned fast lookup, then the staged kernel's error word
    cudaStream_t hstream[2] = {nullptr, nullptr};   // host-path pipeline streams beyond stream and stream2
    int64_t h_buf_cap = 0;
    int64_t stats[6] = {0, 0, 0, 0, 0, 0};
    // kernel timing runs: plain launches with events around the event kernels
    int kernel_timing = 0;
    std::vector<cudaEvent_t> kt_ev;   // 4 per iteration of one sync window
    double kt_ms[3] = {0.0, 0.0, 0.0};
    int64_t kt_count[4] = {0, 0, 0, 0};
    // eigenvalue runs: staging bank, ordered bank, next source, per-history
    // site counts and offsets, per-generation accumulators
    EigenCtl* e_ctl = nullptr;
    FissionSite* e_bank = nullptr;
    int2* e_key = nullptr;
    FissionSite* e_ordered = nullptr;
    int64_t e_bank_cap = 0;
    FissionSite* e_src = nullptr;
    uint32_t* e_count = nullptr;
    unsigned long long* e_off = nullptr;
    unsigned long long* e_tiles = nullptr;
    unsigned long long* e_bad = nullptr;
    int64_t e_n_cap = 0;
    int64_t e_last_M = 0;     // sites in e_ordered after the last generation
};

namespace {

void release_tables(mcx_problem* p)
{
    if (p->tables && --p->tables->refs == 0) delete p->tables;
    p->tables = nullptr;
}

void free_particles(mcx_problem* p)
{
    if (p->p_block) cudaFree(p->p_block);
    p->p_block = nullptr;
    p->P = Particles{};
    p->p_cap = 0;
    p->bins_cap = 0;
}

void drop_graph(mcx_problem* p)
{
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
    p->graph_key.clear();
}

// One device block for the whole particle buffer (SoA arrays + queues + bins).
int ensure_particles(mcx_problem* p, int64_t cap, bool with_w, size_t n_bins, int64_t cum_stride)
{
    if (p->p_block && p->p_cap >= cap && (p->p_has_w || !with_w) && p->bins_cap >= n_bins &&
        p->P.cum_stride >= cum_stride)
        return MCX_OK;
    drop_graph(p);
    int64_t want = cap > p->p_cap ? cap : p->p_cap;
    size_t bins = n_bins > p->bins_cap ? n_bins : p->bins_cap;
    bool w = with_w || p->p_has_w;
    // rows padded to a multiple of 4 entries (32 bytes): the lookup stores
    // four running sums at a time as two 16-byte vectors
    const int64_t cs = ((cum_stride > p->P.cum_stride ? cum_stride : p->P.cum_stride) + 3) & ~(int64_t)3;
    free_particles(p);
    const size_t c = (size_t)want;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t bytes = al(c * 8) * 10 + (w ? al(c * 8 * MCX_MAX_DMAT) : 0) + al(c * 8 * (size_t)cs) + al(c * 8) +
                   al(c * 4) * 3 + al(c * 4) * 3 + al(c) + al(c * 4) * 8 + al((bins + 1) * 4);
    void* blk = nullptr;
    if (simulated_alloc_failure())
        return fail(MCX_ERR_OOM, "particle buffer of %lld slots: simulated failure (MCX_FAIL_ALLOC_AFTER)",
                    (long long)want);
    cudaError_t e = cudaMalloc(&blk, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(MCX_ERR_OOM, "particle buffer of %lld slots (%zu bytes): %s", (long long)want,
                    bytes, cudaGetErrorString(e));
    }
    char* q = (char*)blk;
    auto take = [&](size_t b) {
        char* r = q;
        q += al(b);
        return (void*)r;
    };
    Particles& P = p->P;
    P.cap = want;
    P.stride = want;
    P.x = (double*)take(c * 8);
    P.y = (double*)take(c * 8);
    P.z = (double*)take(c * 8);
    P.u = (double*)take(c * 8);
    P.v = (double*)take(c * 8);
    P.w = (double*)take(c * 8);
    P.E = (double*)take(c * 8);
    P.sig_ta = (double2*)take(c * 16);
    P.sig_nf = (double*)take(c * 8);
    P.W = w ? (double*)take(c * 8 * MCX_MAX_DMAT) : nullptr;
    P.cum = (double*)take(c * 8 * (size_t)cs);
    P.cum_stride = cs;
    P.hist = (int64_t*)take(c * 8);
    P.rng_n = (uint32_t*)take(c * 4);
    P.ncoll = (uint32_t*)take(c * 4);
    P.nsite = (uint32_t*)take(c * 4);
    P.cell = (int32_t*)take(c * 4);
    P.mat = (int32_t*)take(c * 4);
    P.prob = (int32_t*)take(c * 4);
    P.flags = (uint8_t*)take(c);
    for (int k = 0; k < 2; ++k) {
        P.q_xs[k] = (int32_t*)take(c * 4);
        P.q_adv[k] = (int32_t*)take(c * 4);
        P.q_dead[k] = (int32_t*)take(c * 4);
    }
    P.q_coll = (int32_t*)take(c * 4);
    P.q_sorted = (int32_t*)take(c * 4);
    P.bins = (uint32_t*)take((bins + 1) * 4);
    p->p_block = blk;
    p->p_cap = want;
    p->p_has_w = w;
    p->bins_cap = bins;
    return MCX_OK;
}

bool is_finite(double x) { return std::isfinite(x); }

int32_t float_bits(float f)
{
    int32_t b;
    std::memcpy(&b, &f, sizeof(b));
    return b;
}

int validate_desc(const mcx_problem_desc* d)
{
    if (!d) return fail(MCX_ERR_ARG, "desc is NULL");
    if (d->geometry < 0 || d->geometry > MCX_GEOM_NONE)
        return fail(MCX_ERR_ARG, "unknown geometry %d", d->geometry);
    if (d->geometry == MCX_GEOM_NONE) return MCX_OK;
    if (!(d->E0 > 0.0) || !is_finite(d->E0)) return fail(MCX_ERR_ARG, "E0 must be positive and finite");
    if (!(d->E_cut >= 0.0) || !is_finite(d->E_cut)) return fail(MCX_ERR_ARG, "E_cut must be >= 0");
    if (d->n_batches < 1) return fail(MCX_ERR_ARG, "n_batches must be >= 1");
    if (d->n_histories < 1) return fail(MCX_ERR_ARG, "n_histories must be >= 1");
    if ((int64_t)d->n_batches > d->n_histories)
        return fail(MCX_ERR_ARG, "n_batches (%d) exceeds n_histories", d->n_batches);
    if (d->n_histories >= ((int64_t)1 << 40)) return fail(MCX_ERR_ARG, "n_histories too large");
    if (!d->region_material) return fail(MCX_ERR_ARG, "region_material is NULL");
    if (d->geometry == MCX_GEOM_LATTICE) {
        if (d->lattice_n < 1 || d->lattice_n > 4096) return fail(MCX_ERR_ARG, "lattice_n out of range");
        if (!(d->pitch > 0.0) || !is_finite(d->pitch)) return fail(MCX_ERR_ARG, "pitch must be > 0");
        if (!(d->radius > 0.0) || !(2.0 * d->radius < d->pitch))
            return fail(MCX_ERR_ARG, "radius must be in (0, pitch/2)");
        if (!(d->height > 0.0) || !is_finite(d->height)) return fail(MCX_ERR_ARG, "height must be > 0");
        if (d->n_regions != d->lattice_n * d->lattice_n + 1)
            return fail(MCX_ERR_ARG, "lattice needs n^2 + 1 = %d regions, got %d",
                        d->lattice_n * d->lattice_n + 1, d->n_regions);
    } else {
        if (d->n_regions != 1) return fail(MCX_ERR_ARG, "this geometry has exactly 1 region");
    }
    if (d->geometry == MCX_GEOM_SLAB && (!(d->slab_length > 0.0) || !is_finite(d->slab_length)))
        return fail(MCX_ERR_ARG, "slab_length must be > 0");
    if (d->geometry == MCX_GEOM_INFINITE) {
        if (d->n_ebins < 1 || !d->ebin_edges) return fail(MCX_ERR_ARG, "infinite medium needs energy bins");
        for (int i = 0; i <= d->n_ebins; ++i) {
            if (!(d->ebin_edges[i] > 0.0) || !is_finite(d->ebin_edges[i]))
                return fail(MCX_ERR_ARG, "ebin_edges[%d] must be positive and finite", i);
            if (i > 0 && !(d->ebin_edges[i] > d->ebin_edges[i - 1]))
                return fail(MCX_ERR_ARG, "ebin_edges not strictly increasing at %d", i);
        }
    }
    for (int r = 0; r < d->n_regions; ++r)
        if (d->region_material[r] < 0) return fail(MCX_ERR_ARG, "region_material[%d] < 0", r);
    return MCX_OK;
}

int alloc_tallies(mcx_problem* p)
{
    const int64_t B = p->desc.n_batches;
    TRY(dev_alloc(&p->flux, (size_t)(B * p->nb)));
    TRY(dev_alloc(&p->absorb, (size_t)(B * p->nb)));
    TRY(dev_alloc(&p->outcome, (size_t)(B * N_OUT)));
    CUDA_TRY(cudaMemset(p->flux, 0, sizeof(double) * B * p->nb));
    CUDA_TRY(cudaMemset(p->absorb, 0, sizeof(double) * B * p->nb));
    CUDA_TRY(cudaMemset(p->outcome, 0, sizeof(double) * B * N_OUT));
    return MCX_OK;
}

int alloc_derivative_tallies(mcx_problem* p, int M)
{
    dev_free(p->dflux);
    dev_free(p->dabsorb);
    dev_free(p->doutcome);
    p->M = M;
    if (M == 0) return MCX_OK;
    const int64_t B = p->desc.n_batches;
    TRY(dev_alloc(&p->dflux, (size_t)(B * p->nb * M)));
    TRY(dev_alloc(&p->dabsorb, (size_t)(B * p->nb * M)));
    TRY(dev_alloc(&p->doutcome, (size_t)(B * N_OUT * M)));
    CUDA_TRY(cudaMemset(p->dflux, 0, sizeof(double) * B * p->nb * M));
    CUDA_TRY(cudaMemset(p->dabsorb, 0, sizeof(double) * B * p->nb * M));
    CUDA_TRY(cudaMemset(p->doutcome, 0, sizeof(double) * B * N_OUT * M));
    return MCX_OK;
}

int steps_for(int32_t len)
{
    int steps = 0;
    while (len > 1) {
        len -= len >> 1;
        ++steps;
    }
    return steps;
}

int build_hash(TableStore* ts, int32_t H, int sm_count)
{
    dev_free(ts->hidx);
    dev_free(ts->hbound);
    ts->view.H = 0;
    ts->view.hidx = nullptr;
    ts->view.hbound = nullptr;
    ts->view.search_steps = steps_for(ts->max_points - 1);
    if (H == 0) return MCX_OK;
    std::vector<double> hb((size_t)H + 1);
    const double lo = std::log(ts->emin), hi = std::log(ts->emax);
    hb[0] = ts->emin;
    hb[H] = ts->emax;
    for (int b = 1; b < H; ++b) {
        double v = std::exp(lo + (hi - lo) * ((double)b / (double)H));
        if (!(v > hb[b - 1])) v = std::nextafter(hb[b - 1], INFINITY);
        hb[b] = v;
    }
    if (!(hb[H] > hb[H - 1])) return fail(MCX_ERR_ARG, "hash_bins too large for the energy range");
    TRY(dev_alloc(&ts->hbound, (size_t)H + 1));
    TRY(dev_alloc(&ts->hidx, (size_t)ts->view.n_species * ((size_t)H + 1)));
    CUDA_TRY(cudaMemcpy(ts->hbound, hb.data(), sizeof(double) * (H + 1), cudaMemcpyHostToDevice));
    ts->view.H = H;
    ts->view.hbound = ts->hbound;
    ts->view.hash_ln_lo = (float)lo;
    ts->view.hash_scale = (float)((double)H / (hi - lo));
    Tables tmp = ts->view;
    if (launch_build_hash(tmp, ts->hidx, sm_count * 8, 0)) return fail(MCX_ERR_CUDA, "hash build launch failed");
    CUDA_TRY(cudaDeviceSynchronize());
    ts->view.hidx = ts->hidx;
    // fixed step count of the fast path's search: enough for the widest window
    int32_t* d_w = nullptr;
    TRY(dev_alloc(&d_w, 1));
    int32_t one = 1, maxw = 1;
    cudaMemcpy(d_w, &one, 4, cudaMemcpyHostToDevice);
    tmp.hidx = ts->hidx;
    const int lr = launch_hash_max_window(tmp, d_w, sm_count * 8, 0);
    const cudaError_t e = cudaMemcpy(&maxw, d_w, 4, cudaMemcpyDeviceToHost);
    dev_free(d_w);
    if (lr || e != cudaSuccess) return fail(MCX_ERR_CUDA, "hash window scan failed");
    ts->view.search_steps = steps_for(maxw);
    return MCX_OK;
}

int check_handle(const mcx_problem* p)
{
    if (!p) return fail(MCX_ERR_ARG, "problem handle is NULL");
    return MCX_OK;
}

int check_tables(const mcx_problem* p)
{
    TRY(check_handle(p));
    if (!p->tables) return fail(MCX_ERR_STATE, "no cross-section tables loaded");
    return MCX_OK;
}

ProblemDev make_problem_dev(mcx_problem* p, uint64_t seed, int64_t first, bool deriv)
{
    ProblemDev d{};
    const mcx_problem_desc& s = p->desc;
    d.geometry = s.geometry;
    d.lattice_n = s.geometry == MCX_GEOM_LATTICE ? s.lattice_n : 0;
    d.nb = p->nb;
    d.n_batches = s.n_batches;
    d.n_ebins = s.n_ebins;
    d.M = deriv ? p->M : 0;
    d.pitch = s.pitch;
    d.radius = s.radius;
    d.radius2 = s.radius * s.radius;
    d.height = s.height;
    d.slab_length = s.slab_length;
    d.half = 0.5 * (double)d.lattice_n * s.pitch;
    d.E0 = s.E0;
    d.E_cut = s.E_cut;
    d.region_material = p->d_region_material;
    d.lat_plane = p->d_lattice;
    d.lat_centre = p->d_lattice ? p->d_lattice + d.lattice_n + 1 : nullptr;
    d.ebin_edges = p->d_ebin_edges;
    d.key = rng_key(seed, s.problem_id);
    d.n_hist_total = s.n_histories;
    d.first = first;
    d.flux = p->flux;
    d.absorb = p->absorb;
    d.outcome = p->outcome;
    d.dflux = p->dflux;
    d.dabsorb = p->dabsorb;
    d.doutcome = p->doutcome;
    d.ncoll_debug = (s.flags & MCX_FLAG_HISTORY_DEBUG) ? p->ncoll_debug : nullptr;
    return d;
}

int blocks_per_sm(int block)
{
    // the event kernels use <= 64 registers per thread at 1024 threads; keep
    // 2048 resident threads per SM
    int b = 2048 / block;
    return b < 1 ? 1 : b;
}

// What an eigenvalue generation changes in its (single) problem's view.
struct EigenGen {
    int64_t tally_off, n_hist_total;
    const FissionSite* src;
    double k_norm, T_fission;
    FissionSite* bank;
    int2* bank_key;
    int64_t bank_cap;
    uint32_t* site_count;
    EigenCtl* eig;
};

// The event-loop driver shared by mcx_run_batch, mcx_batch_run and the
// generations of mcx_run_eigenvalue (eg != null, one problem).
// Log-energy buckets per material of the event loop's binning of the lookup
// queue (and of the fullest-queue mode's segments): up to this many, as many
// as the shared-memory histogram of 12,288 bins holds for the problem's
// materials (a power of two, at least 16).  On the 17x17 lattice (1e7
// histories, tuned settings) 128 buckets gave 2.204e7 particles/s, 256
// 2.240e7, 512 2.282e7, 1024 2.291e7, 2048 2.242e7.
#ifndef MCX_TRANSPORT_EBUCKETS
#define MCX_TRANSPORT_EBUCKETS 1024
#endif

int transport_ebuckets(int n_materials)
{
    int b = MCX_TRANSPORT_EBUCKETS;
    while (b > 16 && (int64_t)b * (n_materials > 0 ? n_materials : 1) > 12288) b >>= 1;
    return b;
}

int run_loop(mcx_problem* owner, int n_prob, mcx_problem* const* probs, const int64_t* first,
             const int64_t* count, int64_t pif, uint64_t seed, void* user_stream,
             const EigenGen* eg = nullptr)
{
    const TableStore* ts = owner->tables;
    const Tables& t = ts->view;
    if (t.n_ch != 2 && t.n_ch != 3 && t.n_ch != 5)
        return fail(MCX_ERR_ARG, "transport needs 2, 3 or 5 channels");
    if (eg && (n_prob != 1 || t.ch_nu_fission < 0)) return fail(MCX_ERR_ARG, "bad eigenvalue generation");
    const mcx_tune& tu = owner->tune;
    long long total = 0;
    for (int i = 0; i < n_prob; ++i) total += count[i];
    if (pif < 1) return fail(MCX_ERR_ARG, "particles_in_flight must be >= 1");
    if (pif > (int64_t)1 << 30) return fail(MCX_ERR_ARG, "particles_in_flight too large");
    const bool deriv = n_prob == 1 && owner->M > 0;
    int64_t cap = pif < total ? pif : total;
    if (cap < 1) cap = 1;
    LoopConfig c;
    c.mode = tu.mode;
    c.block = tu.block_size;
    c.grid = owner->sm_count * blocks_per_sm(tu.block_size);
    c.sort_period = tu.mode != MCX_QUEUELESS ? tu.sort_period : 0;
    c.sort_threshold = tu.sort_threshold;
    c.n_ebuckets = transport_ebuckets(t.n_materials);
    c.n_sort_bins = t.n_materials * c.n_ebuckets;
    c.sort_ln_lo = (float)std::log(ts->emin);
    c.sort_scale = (float)((double)c.n_ebuckets / (std::log(ts->emax) - std::log(ts->emin)));
    c.derivatives = deriv ? owner->M : 0;
    c.eigen = eg ? 1 : 0;
    if ((size_t)c.n_sort_bins * 4 > 48 * 1024) c.sort_period = 0;  // bins must fit shared memory
    TRY(ensure_particles(owner, cap, deriv, (size_t)c.n_sort_bins, t.max_mat_species));
    // the buffer may be larger than this run needs: use exactly `cap` slots
    owner->P.cap = cap;
    // problems and work offsets
    if (owner->probs_cap < n_prob) {
        drop_graph(owner);
        dev_free(owner->d_probs);
        dev_free(owner->d_work_off);
        owner->probs_cap = 0;   // stays 0 if an allocation below fails
        TRY(dev_alloc(&owner->d_probs, (size_t)n_prob));
        TRY(dev_alloc(&owner->d_work_off, (size_t)n_prob + 1));
        owner->probs_cap = n_prob;
    }
    std::vector<ProblemDev> hp((size_t)n_prob);
    std::vector<int64_t> wo((size_t)n_prob + 1, 0);
    for (int i = 0; i < n_prob; ++i) {
        mcx_problem* q = probs[i];
        if (q->desc.flags & MCX_FLAG_HISTORY_DEBUG) {
            if (q->debug_cap < count[i]) {
                dev_free(q->ncoll_debug);
                q->debug_cap = 0;
                TRY(dev_alloc(&q->ncoll_debug, (size_t)count[i]));
                q->debug_cap = count[i];
            }
            q->debug_n = count[i];
        }
        hp[i] = make_problem_dev(q, seed, first[i], deriv);
        wo[i + 1] = wo[i] + count[i];
    }
    if (eg) {
        ProblemDev& d = hp[0];
        d.tally_off = eg->tally_off;
        d.n_hist_total = eg->n_hist_total;
        d.src = eg->src;
        d.k_norm = eg->k_norm;
        d.T_fission = eg->T_fission;
        d.bank = eg->bank;
        d.bank_key = eg->bank_key;
        d.bank_cap = eg->bank_cap;
        d.site_count = eg->site_count;
        d.eig = eg->eig;
    }
    cudaStream_t us = (cudaStream_t)user_stream;
    cudaStream_t st = owner->stream;
    CUDA_TRY(cudaEventRecord(owner->ev_a, us));
    CUDA_TRY(cudaStreamWaitEvent(st, owner->ev_a, 0));
    CUDA_TRY(cudaMemcpyAsync(owner->d_probs, hp.data(), sizeof(ProblemDev) * n_prob,
                             cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(owner->d_work_off, wo.data(), sizeof(int64_t) * (n_prob + 1),
                             cudaMemcpyHostToDevice, st));
    const long long max_iters = tu.max_event_iters > 0 ? tu.max_event_iters : 4000000LL;
    if (launch_run_init(c, owner->P, owner->d_ctl, total, n_prob, max_iters, st))
        return fail(MCX_ERR_CUDA, "run init launch failed");
    const int K = tu.iters_per_sync;
    // graph key: everything the captured kernels see by value
    std::vector<unsigned char> key;
    auto put = [&](const void* v, size_t n) {
        key.insert(key.end(), (const unsigned char*)v, (const unsigned char*)v + n);
    };
    put(&c, sizeof(c));
    put(&t, sizeof(t));
    put(&owner->P, sizeof(Particles));
    put(&owner->d_probs, sizeof(void*));
    put(&owner->d_work_off, sizeof(void*));
    put(&K, sizeof(K));
    int kernels_per_iter = 0;
    if (tu.use_graph) {
        if (!owner->gexec || owner->graph_key != key) {
            drop_graph(owner);
            cudaGraph_t g = nullptr;
            CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            int bad = 0;
            for (int k = 0; k < K; ++k) {
                const int r = launch_iteration(c, t, owner->P, owner->d_probs, owner->d_work_off,
                                               owner->d_ctl, st);
                if (r < 0) bad = 1;
                kernels_per_iter = r;
            }
            cudaError_t ec = cudaStreamEndCapture(st, &g);
            if (bad || ec != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                return fail(MCX_ERR_CUDA, "capturing the event loop failed: %s", cudaGetErrorString(ec));
            }
            cudaError_t ei = cudaGraphInstantiate(&owner->gexec, g, 0);
            cudaGraphDestroy(g);
            if (ei != cudaSuccess) {
                owner->gexec = nullptr;
                return fail(MCX_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ei));
            }
            owner->graph_key = key;
        }
    }
    if (kernels_per_iter == 0) {
        const bool sorting = c.mode != MCX_QUEUELESS && c.sort_period > 0;
        kernels_per_iter = 5 + (sorting ? 4 : 0);   // one binned queue per iteration or step
    }
    int64_t launches = 0, kernels = 0;
    const int64_t max_launches = max_iters / K + 4;
    int status = MCX_OK;
    const bool timing = owner->kernel_timing != 0;
    if (timing) {
        while ((int)owner->kt_ev.size() < 4 * K) {
            cudaEvent_t e = nullptr;
            CUDA_TRY(cudaEventCreate(&e));
            owner->kt_ev.push_back(e);
        }
        for (int e = 0; e < 3; ++e) owner->kt_ms[e] = 0.0;
    }
    const auto t_start = std::chrono::steady_clock::now();
    for (;;) {
        if (tu.use_graph && !timing) {
            CUDA_TRY(cudaGraphLaunch(owner->gexec, st));
        } else {
            for (int k = 0; k < K; ++k)
                if (launch_iteration(c, t, owner->P, owner->d_probs, owner->d_work_off, owner->d_ctl, st,
                                     timing ? owner->kt_ev.data() + 4 * k : nullptr) < 0)
                    return fail(MCX_ERR_CUDA, "event kernel launch failed");
        }
        ++launches;
        kernels += (int64_t)K * kernels_per_iter;
        CUDA_TRY(cudaMemcpyAsync(owner->h_ctl, owner->d_ctl, sizeof(RunCtl), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        if (timing) {
            for (int k = 0; k < K; ++k)
                for (int e = 0; e < 3; ++e) {
                    float ms = 0.f;
                    CUDA_TRY(cudaEventElapsedTime(&ms, owner->kt_ev[4 * k + e], owner->kt_ev[4 * k + e + 1]));
                    owner->kt_ms[e] += ms;
                }
        }
        if (owner->h_ctl->error) {
            if (owner->h_ctl->error == MCX_ERR_ITER_LIMIT)
                status = fail(MCX_ERR_ITER_LIMIT, "event loop reached its cap of %lld iterations",
                              (long long)max_iters);
            else if (owner->h_ctl->error == MCX_ERR_BOUNDS)
                status = bounds_failure(bounds_error_transport(), "transport");
            else
                status = fail(owner->h_ctl->error, "device error %d", owner->h_ctl->error);
            break;
        }
        if (owner->h_ctl->done) break;
        if (tu.time_limit_s > 0.0 &&
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count() > tu.time_limit_s) {
            status = fail(MCX_ERR_TIMEOUT, "run exceeded its time limit of %.3f s after %lld iterations",
                          tu.time_limit_s, (long long)owner->h_ctl->iters);
            break;
        }
        if (launches >= max_launches) {
            status = fail(MCX_ERR_ITER_LIMIT, "host loop reached its launch cap");
            break;
        }
    }
    owner->stats[0] = owner->h_ctl->iters;
    owner->stats[1] = launches;
    owner->stats[2] = kernels;
    for (int e = 0; e < 3; ++e)
        owner->stats[3 + e] = c.mode == MCX_QUEUED_FULLEST ? owner->h_ctl->sel_count[e] : 0;
    for (int e = 0; e < 4; ++e) owner->kt_count[e] = c.mode == MCX_QUEUED ? owner->h_ctl->ev_count[e] : -1;
    CUDA_TRY(cudaEventRecord(owner->ev_b, st));
    CUDA_TRY(cudaStreamWaitEvent(us, owner->ev_b, 0));
    return status;
}

int lookup_grid(const mcx_problem* p) { return p->sm_count * 8; }

int ensure_lookup_scratch(mcx_problem* p, int64_t n, size_t)
{
    if (p->perm_cap < n) {
        dev_free(p->perm);
        p->perm_cap = 0;
        TRY(dev_alloc(&p->perm, (size_t)n));
        p->perm_cap = n;
    }
    return MCX_OK;
}

// Binning of a batch of n lookups (about kLookupsPerBucket lookups per
// material and log-energy bucket), at most max_bins bins.
SortParams batch_sort_params(const TableStore* ts, int64_t n, int64_t max_bins = (int64_t)1 << 21,
                             int64_t per_bucket = kLookupsPerBucket)
{
    return lookup_sort_params(ts->view.n_materials, ts->emin, ts->emax, n, max_bins, per_bucket);
}

// Bin lookups into perm (device, [n]), about per_bucket lookups per bin;
// bins scratch owned by the problem.  With Eb and Mb (device, [n]) also the
// energies and materials in the binned order: carried through the two-level
// passes, or gathered after the one-level sort.
int sort_device(mcx_problem* p, int64_t n, const double* E, const int32_t* mat, int32_t* perm,
                cudaStream_t st, int64_t per_bucket = kLookupsPerBucket, double* Eb = nullptr,
                int32_t* Mb = nullptr)
{
    const bool carry = Eb != nullptr && Mb != nullptr;
    const SortParams sp = batch_sort_params(p->tables, n, (int64_t)1 << 21, per_bucket);
    // large batches: the two-level binning (no global atomic per lookup)
    const bool two = n >= kBin2MinLookups;
    const size_t nb = two ? lookup_sort2_place_words(sp, n)
                          : (size_t)sp.n_materials * sp.n_ebuckets + 1 + kSortScanParts;
    if (p->lbins_cap < nb) {
        dev_free(p->lbins);
        p->lbins_cap = 0;
        TRY(dev_alloc(&p->lbins, nb));
        p->lbins_cap = nb;
    }
    if (two) {
        // keys, indices, fine bins; with a carry then (from an even word, for
        // 8-byte alignment) the coarse-order energies
        const size_t base = 2 * (size_t)n + ((size_t)n + 1) / 2;
        const size_t e_off = (base + 1) & ~(size_t)1;
        const size_t words = carry ? e_off + 2 * (size_t)n : base;
        if (p->bin2_cap < words) {
            dev_free(p->bin2);
            p->bin2_cap = 0;
            TRY(dev_alloc(&p->bin2, words));
            p->bin2_cap = words;
        }
        const Bin2Carry cy{reinterpret_cast<double*>(p->bin2 + e_off), Eb, Mb};
        const int r = launch_lookup_sort2(sp, n, E, mat, p->lbins, reinterpret_cast<uint32_t*>(p->bin2),
                                          p->bin2 + n, reinterpret_cast<uint16_t*>(p->bin2 + 2 * n), perm,
                                          p->sm_count, st, carry ? &cy : nullptr);
        if (r == 0) return MCX_OK;
        if (r == -1) return fail(MCX_ERR_CUDA, "lookup binning launch failed");
        // r == -2: too many tiles x coarse bins; the one-level sort below
        const size_t nb1 = (size_t)sp.n_materials * sp.n_ebuckets + 1 + kSortScanParts;
        if (p->lbins_cap < nb1) {
            dev_free(p->lbins);
            p->lbins_cap = 0;
            TRY(dev_alloc(&p->lbins, nb1));
            p->lbins_cap = nb1;
        }
    }
    if (launch_lookup_sort(sp, n, E, mat, p->lbins, perm, lookup_grid(p), st))
        return fail(MCX_ERR_CUDA, "lookup sort launch failed");
    if (carry && launch_gather_inputs(n, perm, E, mat, sp.n_materials, Eb, Mb, lookup_grid(p), st))
        return fail(MCX_ERR_CUDA, "input gather launch failed");
    return MCX_OK;
}

// Chunk counters of in-order sweeps over binned orders (one per stream that
// may run a binned lookup: the device paths use counter 0, the host path one
// per pipeline slot), then the staged lookup kernel's error word.
int ensure_work_ctr(mcx_problem* p)
{
    if (!p->work_ctr) {
        TRY(dev_alloc(&p->work_ctr, kWorkCtrs + 1));
        CUDA_TRY(cudaMemset(p->work_ctr, 0, (kWorkCtrs + 1) * sizeof(unsigned long long)));
    }
    return MCX_OK;
}

// Lookup on device buffers, queued on `st`, in the order `perm` (or natural).
// A binned order (perm != nullptr) on the fast path is swept in order by
// warps claiming chunks from a counter (slot `ctr` of the problem's two),
// with one resident grid of blocks.
int lookup_device_ordered(mcx_problem* p, int64_t n, const double* E, const int32_t* mat,
                          const int32_t* perm, void* out, int32_t flags, cudaStream_t st,
                          int ctr = 0)
{
    const bool out32 = (flags & MCX_LOOKUP_OUT32) != 0;
    const TableStore* ts = p->tables;
    unsigned long long* work = nullptr;
    if (perm && (flags & MCX_LOOKUP_FAST)) {
        TRY(ensure_work_ctr(p));
        work = p->work_ctr + ctr;
    }
    int r = -2;
    if (work && (flags & MCX_LOOKUP_STAGED))
        r = launch_xs_lookup_staged(ts->view, batch_sort_params(ts, n), n, E, mat, perm, out, out32,
                                    p->sm_count, st, work,
                                    reinterpret_cast<unsigned int*>(p->work_ctr + kWorkCtrs));
    if (r == -2) {
        const int grid =
            work ? p->sm_count * ((flags & MCX_LOOKUP_LINEAR) ? kLinBlocksPerSm : kFastBlocksPerSm) : lookup_grid(p);
        r = (flags & MCX_LOOKUP_FAST)
                ? launch_xs_lookup_fast(ts->view, n, E, mat, perm, out, out32, grid, st, work,
                                        (flags & MCX_LOOKUP_LINEAR) != 0, (flags & MCX_LOOKUP_BINNED_INPUTS) != 0)
                : launch_xs_lookup_exact(ts->view, n, E, mat, perm, static_cast<double*>(out), lookup_grid(p), st);
    }
    if (r) return fail(MCX_ERR_CUDA, "lookup launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return MCX_OK;
}

// Lookup on device buffers, queued on `st` (binned first with MCX_LOOKUP_SORT).
int lookup_device(mcx_problem* p, int64_t n, const double* E, const int32_t* mat, void* out,
                  int32_t flags, cudaStream_t st)
{
    const int32_t* perm = nullptr;
    const int32_t pass = flags & (MCX_LOOKUP_FAST | MCX_LOOKUP_STAGED | MCX_LOOKUP_OUT32 | MCX_LOOKUP_LINEAR);
    if (flags & MCX_LOOKUP_SORT) {
        TRY(ensure_lookup_scratch(p, n, 0));
        // large fast batches: the binning hands the inputs over in the binned
        // order, and the lookup reads them in sequence (the same results)
        if ((flags & MCX_LOOKUP_FAST) && !(flags & MCX_LOOKUP_STAGED) && n >= kBin2MinLookups) {
            if (p->bin_in_cap < n) {
                dev_free(p->bin_E);
                dev_free(p->bin_M);
                p->bin_in_cap = 0;
                TRY(dev_alloc(&p->bin_E, (size_t)n));
                TRY(dev_alloc(&p->bin_M, (size_t)n));
                p->bin_in_cap = n;
            }
            TRY(sort_device(p, n, E, mat, p->perm, st, kLookupsPerBucket, p->bin_E, p->bin_M));
            return lookup_device_ordered(p, n, p->bin_E, p->bin_M, p->perm, out, pass | MCX_LOOKUP_BINNED_INPUTS, st);
        }
        TRY(sort_device(p, n, E, mat, p->perm, st));
        perm = p->perm;
    }
    return lookup_device_ordered(p, n, E, mat, perm, out, pass, st);
}

// Eigenvalue scratch: per-history arrays for N histories and a staging and
// an ordered bank of `bank_cap` sites (grown, never shrunk).
int ensure_eigen(mcx_problem* p, int64_t N, int64_t bank_cap)
{
    if (!p->e_ctl) TRY(dev_alloc(&p->e_ctl, 1));
    if (!p->e_bad) TRY(dev_alloc(&p->e_bad, 1));
    if (p->e_n_cap < N) {
        dev_free(p->e_src);
        dev_free(p->e_count);
        dev_free(p->e_off);
        dev_free(p->e_tiles);
        p->e_n_cap = 0;
        TRY(dev_alloc(&p->e_src, (size_t)N));
        TRY(dev_alloc(&p->e_count, (size_t)N));
        TRY(dev_alloc(&p->e_off, (size_t)N));
        TRY(dev_alloc(&p->e_tiles, (size_t)bank_scan_tiles(N) + 1));
        p->e_n_cap = N;
    }
    if (p->e_bank_cap < bank_cap) {
        dev_free(p->e_bank);
        dev_free(p->e_key);
        dev_free(p->e_ordered);
        p->e_bank_cap = 0;
        p->e_last_M = 0;
        TRY(dev_alloc(&p->e_bank, (size_t)bank_cap));
        TRY(dev_alloc(&p->e_key, (size_t)bank_cap));
        TRY(dev_alloc(&p->e_ordered, (size_t)bank_cap));
        p->e_bank_cap = bank_cap;
    }
    return MCX_OK;
}

}  // namespace

// Read-only view of a problem's lookup tables for other translation units of
// the library (the static-scratch entry point).  Returns MCX_OK or an error.
namespace mcx {
int problem_lookup_view(const mcx_problem* p, LookupView* v)
{
    TRY(check_tables(p));
    const TableStore* ts = p->tables;
    v->tables = ts->view;
    v->sort = batch_sort_params(ts, MCX_STATIC_MAX_LOOKUPS, MCX_STATIC_MAX_BINS);
    v->emin = ts->emin;
    v->emax = ts->emax;
    v->device = p->device;
    v->grid = lookup_grid(p);
    v->sm_count = p->sm_count;
    return MCX_OK;
}
int set_error(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace mcx

// ===================================================================== ABI

extern "C" {

const char* mcx_last_error(void) { return g_err.c_str(); }

const char* mcx_version(void) { return "libmcx 0.1 (sm_103a)"; }

void mcx_default_tuning(mcx_tune* t)
{
    if (!t) return;
    t->mode = MCX_QUEUELESS;
    t->block_size = 256;
    t->sort_period = 0;
    t->sort_threshold = 20000;
    t->iters_per_sync = 16;
    t->max_event_iters = 0;
    t->use_graph = 1;
    t->time_limit_s = 0.0;
}

int mcx_init_problem(const mcx_problem_desc* desc, mcx_problem** out)
{
    g_err.clear();
    if (!out) return fail(MCX_ERR_ARG, "out is NULL");
    *out = nullptr;
    TRY(validate_desc(desc));
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (desc->device < 0 || desc->device >= ndev)
        return fail(MCX_ERR_ARG, "device %d not present (%d devices)", desc->device, ndev);
    DeviceGuard dg(desc->device);
    if (!dg.ok) return fail(MCX_ERR_CUDA, "cudaSetDevice(%d) failed", desc->device);
    mcx_problem* p = new (std::nothrow) mcx_problem();
    if (!p) return fail(MCX_ERR_OOM, "host allocation failed");
    p->desc = *desc;
    p->device = desc->device;
    p->sm_count = sm_count_of(desc->device);
    mcx_default_tuning(&p->tune);
    int rc = MCX_OK;
    auto bail = [&](int code) {
        mcx_destroy(p);
        return code;
    };
    if (desc->geometry != MCX_GEOM_NONE) {
        p->region_material.assign(desc->region_material, desc->region_material + desc->n_regions);
        if (desc->geometry == MCX_GEOM_INFINITE)
            p->ebin_edges.assign(desc->ebin_edges, desc->ebin_edges + desc->n_ebins + 1);
        p->desc.region_material = p->region_material.data();
        p->desc.ebin_edges = p->ebin_edges.empty() ? nullptr : p->ebin_edges.data();
        p->nb = desc->geometry == MCX_GEOM_INFINITE ? desc->n_ebins
                : desc->geometry == MCX_GEOM_LATTICE ? desc->n_regions
                                                     : 1;
        if ((rc = dev_alloc(&p->d_region_material, p->region_material.size())) != MCX_OK) return bail(rc);
        if (cudaMemcpy(p->d_region_material, p->region_material.data(),
                       sizeof(int32_t) * p->region_material.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(fail(MCX_ERR_CUDA, "copying region materials failed"));
        if (desc->geometry == MCX_GEOM_LATTICE) {
            // cell planes -half + pitch i (i = 0..n) and centres
            // -half + pitch (i + 0.5), the FP64 expressions the kernels
            // would otherwise evaluate every flight (same values, bit for bit)
            const int32_t n = desc->lattice_n;
            const double half = 0.5 * (double)n * desc->pitch;
            std::vector<double> lat((size_t)2 * n + 1);
            for (int32_t i = 0; i <= n; ++i) lat[i] = -half + desc->pitch * (double)i;
            for (int32_t i = 0; i < n; ++i) lat[n + 1 + i] = -half + desc->pitch * ((double)i + 0.5);
            if ((rc = dev_alloc(&p->d_lattice, lat.size())) != MCX_OK) return bail(rc);
            if (cudaMemcpy(p->d_lattice, lat.data(), sizeof(double) * lat.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess)
                return bail(fail(MCX_ERR_CUDA, "copying lattice coordinates failed"));
        }
        if (!p->ebin_edges.empty()) {
            if ((rc = dev_alloc(&p->d_ebin_edges, p->ebin_edges.size())) != MCX_OK) return bail(rc);
            if (cudaMemcpy(p->d_ebin_edges, p->ebin_edges.data(), sizeof(double) * p->ebin_edges.size(),
                           cudaMemcpyHostToDevice) != cudaSuccess)
                return bail(fail(MCX_ERR_CUDA, "copying energy bins failed"));
        }
        if ((rc = alloc_tallies(p)) != MCX_OK) return bail(rc);
    } else {
        p->desc.region_material = nullptr;
        p->desc.ebin_edges = nullptr;
    }
    if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->stream2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_a, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_b, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(MCX_ERR_CUDA, "stream/event creation failed"));
    if ((rc = dev_alloc(&p->d_ctl, 1)) != MCX_OK) return bail(rc);
    if (cudaMallocHost((void**)&p->h_ctl, sizeof(RunCtl)) != cudaSuccess)
        return bail(fail(MCX_ERR_OOM, "pinned host allocation failed"));
    memset(p->h_ctl, 0, sizeof(RunCtl));
    *out = p;
    return MCX_OK;
}

void mcx_destroy(mcx_problem* p)
{
    if (!p) return;
    DeviceGuard dg(p->device);
    if (p->stream) cudaStreamSynchronize(p->stream);
    for (cudaEvent_t e : p->kt_ev) cudaEventDestroy(e);
    p->kt_ev.clear();
    drop_graph(p);
    release_tables(p);
    free_particles(p);
    dev_free(p->d_region_material);
    dev_free(p->d_lattice);
    dev_free(p->d_ebin_edges);
    dev_free(p->flux);
    dev_free(p->absorb);
    dev_free(p->outcome);
    dev_free(p->dflux);
    dev_free(p->dabsorb);
    dev_free(p->doutcome);
    dev_free(p->d_probs);
    dev_free(p->d_work_off);
    dev_free(p->d_ctl);
    dev_free(p->ncoll_debug);
    dev_free(p->perm);
    dev_free(p->bin_E);
    dev_free(p->bin_M);
    dev_free(p->lbins);
    dev_free(p->bin2);
    dev_free(p->h_buf);
    dev_free(p->work_ctr);
    dev_free(p->e_ctl);
    dev_free(p->e_bank);
    dev_free(p->e_key);
    dev_free(p->e_ordered);
    dev_free(p->e_src);
    dev_free(p->e_count);
    dev_free(p->e_off);
    dev_free(p->e_tiles);
    dev_free(p->e_bad);
    if (p->h_ctl) cudaFreeHost(p->h_ctl);
    if (p->ev_a) cudaEventDestroy(p->ev_a);
    if (p->ev_b) cudaEventDestroy(p->ev_b);
    if (p->stream) cudaStreamDestroy(p->stream);
    if (p->stream2) cudaStreamDestroy(p->stream2);
    for (cudaStream_t& hs : p->hstream)
        if (hs) cudaStreamDestroy(hs);
    delete p;
}

int mcx_load_xs_tables(mcx_problem* p, int32_t n_species, const int64_t* goff, const double* energies,
                       const double* sigma, int32_t n_ch, const double* awr, int32_t n_materials,
                       const int32_t* moff, const int32_t* msp, const double* mden,
                       int32_t precision, int32_t hash_bins)
{
    g_err.clear();
    TRY(check_handle(p));
    if (n_species < 1) return fail(MCX_ERR_ARG, "n_species must be >= 1");
    if (n_ch < 1 || n_ch > 5) return fail(MCX_ERR_ARG, "n_ch must be in 1..5");
    if (!goff || !energies || !sigma || !awr || !moff || !msp || !mden)
        return fail(MCX_ERR_ARG, "NULL table pointer");
    if (precision != MCX_FP64 && precision != MCX_FP32) return fail(MCX_ERR_ARG, "unknown precision");
    if (hash_bins < 0 || hash_bins > 10000000) return fail(MCX_ERR_ARG, "hash_bins out of range");
    if (n_materials < 1) return fail(MCX_ERR_ARG, "n_materials must be >= 1");
    if (goff[0] != 0) return fail(MCX_ERR_ARG, "grid_offsets[0] must be 0");
    for (int s = 0; s < n_species; ++s)
        if (goff[s + 1] - goff[s] < 2) return fail(MCX_ERR_ARG, "species %d has fewer than 2 points", s);
    const int64_t P = goff[n_species];
    if (P >= ((int64_t)1 << 31)) return fail(MCX_ERR_ARG, "too many grid points");
    double emin = INFINITY, emax = -INFINITY;
    for (int s = 0; s < n_species; ++s) {
        for (int64_t i = goff[s]; i < goff[s + 1]; ++i) {
            const double e = energies[i];
            if (!(e > 0.0) || !is_finite(e))
                return fail(MCX_ERR_ARG, "energies[%lld] must be positive and finite", (long long)i);
            if (i > goff[s] && !(e > energies[i - 1]))
                return fail(MCX_ERR_ARG, "grid of species %d not strictly increasing at point %lld", s,
                            (long long)i);
        }
        emin = std::fmin(emin, energies[goff[s]]);
        emax = std::fmax(emax, energies[goff[s + 1] - 1]);
        if (!(awr[s] >= 1.0) || !is_finite(awr[s])) return fail(MCX_ERR_ARG, "awr[%d] must be >= 1", s);
    }
    for (int64_t i = 0; i < P * n_ch; ++i) {
        if (!(sigma[i] >= 0.0) || !is_finite(sigma[i]))
            return fail(MCX_ERR_ARG, "sigma[%lld] must be finite and >= 0", (long long)i);
        if (precision == MCX_FP32 && !(sigma[i] <= 3.4028234663852886e38))
            return fail(MCX_ERR_ARG, "sigma[%lld] exceeds the FP32 range", (long long)i);
    }
    if (moff[0] != 0) return fail(MCX_ERR_ARG, "mat_offsets[0] must be 0");
    int32_t maxs = 0;
    for (int m = 0; m < n_materials; ++m) {
        const int32_t c = moff[m + 1] - moff[m];
        if (c < 1) return fail(MCX_ERR_ARG, "material %d has no species", m);
        if (c > maxs) maxs = c;
    }
    const int64_t nnz = moff[n_materials];
    for (int64_t i = 0; i < nnz; ++i) {
        if (msp[i] < 0 || msp[i] >= n_species)
            return fail(MCX_ERR_ARG, "mat_species[%lld] = %d out of range", (long long)i, msp[i]);
        if (!(mden[i] >= 0.0) || !is_finite(mden[i]))
            return fail(MCX_ERR_ARG, "mat_dens[%lld] must be finite and >= 0", (long long)i);
    }
    if (p->desc.geometry != MCX_GEOM_NONE) {
        for (size_t r = 0; r < p->region_material.size(); ++r)
            if (p->region_material[r] >= n_materials)
                return fail(MCX_ERR_ARG, "region_material[%zu] = %d >= n_materials", r, p->region_material[r]);
        if ((p->desc.flags & MCX_FLAG_DERIVATIVES) && n_materials > MCX_MAX_DMAT)
            return fail(MCX_ERR_ARG, "derivative tallies support at most %d materials", MCX_MAX_DMAT);
    }
    DeviceGuard dg(p->device);
    if (p->stream) CUDA_TRY(cudaStreamSynchronize(p->stream));
    TableStore* ts = new (std::nothrow) TableStore();
    if (!ts) return fail(MCX_ERR_OOM, "host allocation failed");
    ts->device = p->device;
    auto bail = [&](int code) {
        delete ts;
        return code;
    };
    int rc;
    // fast-path copies: per material entry {first point, points, species,
    // FP32 density}; per point a 16-byte aligned record {g_hi, g_lo, sigma...}
    std::vector<int4> ment((size_t)nnz);
    int32_t max_points = 0;
    for (int64_t i = 0; i < nnz; ++i) {
        const int32_t sp = msp[i];
        ment[i] = make_int4((int32_t)goff[sp], (int32_t)(goff[sp + 1] - goff[sp]), sp,
                            float_bits((float)mden[i]));
    }
    for (int s2 = 0; s2 < n_species; ++s2)
        if (goff[s2 + 1] - goff[s2] > max_points) max_points = (int32_t)(goff[s2 + 1] - goff[s2]);
    // reciprocal interval widths for the transport lookup's fraction (0 after
    // a species' last point, which never starts an interval)
    std::vector<double> winv((size_t)P, 0.0);
    for (int32_t s2 = 0; s2 < n_species; ++s2)
        for (int64_t k = goff[s2]; k + 1 < goff[s2 + 1]; ++k) winv[k] = 1.0 / (energies[k + 1] - energies[k]);
    // fast-path point records {g_hi, g_lo, sigma_0 .. sigma_{n_ch-1}, ...};
    // two-float4 records end with the FP32 reciprocal interval width
    const int frec_w = n_ch <= 2 ? 1 : 2;
    std::vector<float> rec((size_t)P * 4 * frec_w, 0.f);
    for (int64_t i = 0; i < P; ++i) {
        float* r = &rec[(size_t)i * 4 * frec_w];
        const float hi = (float)energies[i];
        r[0] = hi;
        r[1] = (float)(energies[i] - (double)hi);
        for (int c = 0; c < n_ch; ++c) r[2 + c] = (float)sigma[i * n_ch + c];
        if (frec_w == 2) r[7] = (float)winv[i];
    }
    // elastic kinematics: E' = E (A^2 + 2 A mu + 1) / (A + 1)^2 multiplies by this
    std::vector<double> inv_a1sq((size_t)n_species);
    for (int32_t s2 = 0; s2 < n_species; ++s2) inv_a1sq[s2] = 1.0 / ((awr[s2] + 1.0) * (awr[s2] + 1.0));
    // two padding entries past the last energy: the staged lookup copies FP64
    // energies in 16-byte pairs and may read one entry past a species' end
    if ((rc = dev_alloc(&ts->goff, (size_t)n_species + 1)) || (rc = dev_alloc(&ts->E, (size_t)P + 2)) ||
        (rc = dev_alloc(&ts->winv, (size_t)P)) || (rc = dev_alloc(&ts->slope, (size_t)P * n_ch)) ||
        (rc = dev_alloc(&ts->ttot, (size_t)P)) ||
        (rc = dev_alloc(&ts->tpair, (size_t)P * (n_ch == 2 ? 3 : 4))) || (rc = dev_alloc(&ts->mden2, (size_t)nnz)) ||
        (rc = dev_alloc(&ts->frec, (size_t)P * frec_w)) ||
        (rc = dev_alloc(&ts->awr, (size_t)n_species)) || (rc = dev_alloc(&ts->inv_a1sq, (size_t)n_species)) || (rc = dev_alloc(&ts->moff, (size_t)n_materials + 1)) ||
        (rc = dev_alloc(&ts->msp, (size_t)nnz)) || (rc = dev_alloc(&ts->mden, (size_t)nnz)) ||
        (rc = dev_alloc(&ts->ment, (size_t)nnz)))
        return bail(rc);
    const size_t sig_bytes = (size_t)P * n_ch * (precision == MCX_FP32 ? 4 : 8);
    if (simulated_alloc_failure() || cudaMalloc(&ts->sigma, sig_bytes) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(MCX_ERR_OOM, "sigma table of %zu bytes", sig_bytes));
    }
    bool ok = cudaMemcpy(ts->goff, goff, 8 * (n_species + 1), cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(ts->E, energies, 8 * P, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemset(ts->E + P, 0x7f, 16) == cudaSuccess &&
              cudaMemcpy(ts->winv, winv.data(), 8 * P, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(ts->frec, rec.data(), sizeof(float) * rec.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(ts->awr, awr, 8 * n_species, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(ts->inv_a1sq, inv_a1sq.data(), 8 * n_species, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(ts->moff, moff, 4 * (n_materials + 1), cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(ts->msp, msp, 4 * nnz, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(ts->mden, mden, 8 * nnz, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(ts->ment, ment.data(), sizeof(int4) * nnz, cudaMemcpyHostToDevice) == cudaSuccess;
    if (ok) {
        if (precision == MCX_FP32) {
            std::vector<float> s32((size_t)P * n_ch);
            for (size_t i = 0; i < s32.size(); ++i) s32[i] = (float)sigma[i];
            ok = cudaMemcpy(ts->sigma, s32.data(), sig_bytes, cudaMemcpyHostToDevice) == cudaSuccess;
        } else {
            ok = cudaMemcpy(ts->sigma, sigma, sig_bytes, cudaMemcpyHostToDevice) == cudaSuccess;
        }
    }
    if (!ok) return bail(fail(MCX_ERR_CUDA, "uploading tables failed"));
    Tables& v = ts->view;
    v.n_species = n_species;
    v.n_ch = n_ch;
    v.precision = precision;
    v.n_materials = n_materials;
    v.max_mat_species = maxs;
    v.ch_scatter = n_ch == 5 ? 1 : 0;
    v.ch_absorb = n_ch == 5 ? 2 : 1;
    v.ch_nu_fission = n_ch == 5 ? 4 : (n_ch == 3 ? 2 : -1);
    v.n_points = P;
    v.goff = ts->goff;
    v.E = ts->E;
    v.winv = ts->winv;
    v.slope = ts->slope;
    v.ttot = ts->ttot;
    v.tpair = ts->tpair;
    v.tpair_w = n_ch == 2 ? 3 : 4;
    v.mden2 = ts->mden2;
    v.frec = ts->frec;
    v.frec_w = frec_w;
    v.sigma = ts->sigma;
    v.awr = ts->awr;
    v.inv_a1sq = ts->inv_a1sq;
    v.moff = ts->moff;
    v.msp = ts->msp;
    v.mden = ts->mden;
    v.ment = ts->ment;
    ts->h_ment = ment;
    ts->max_points = max_points;
    ts->emin = emin;
    ts->emax = emax;
    ts->nnz = nnz;
    ts->h_moff.assign(moff, moff + n_materials + 1);
    if (launch_build_slopes(v, ts->slope, ts->ttot, p->sm_count * 8, nullptr) ||
        launch_build_pairs(v, ts->tpair, ts->mden2, ts->nnz ? ts->nnz : nnz, p->sm_count * 8, nullptr) ||
        cudaDeviceSynchronize() != cudaSuccess)
        return bail(fail(MCX_ERR_CUDA, "slope table build failed"));
    if ((rc = build_hash(ts, hash_bins, p->sm_count)) != MCX_OK) return bail(rc);
    drop_graph(p);
    release_tables(p);
    p->tables = ts;
    if (p->desc.geometry != MCX_GEOM_NONE)
        TRY(alloc_derivative_tallies(p, (p->desc.flags & MCX_FLAG_DERIVATIVES) ? n_materials : 0));
    return MCX_OK;
}

int mcx_share_xs_tables(mcx_problem* dst, const mcx_problem* src)
{
    g_err.clear();
    TRY(check_handle(dst));
    TRY(check_tables(src));
    if (dst->device != src->device) return fail(MCX_ERR_ARG, "problems live on different devices");
    TableStore* ts = src->tables;
    if (dst->desc.geometry != MCX_GEOM_NONE) {
        for (size_t r = 0; r < dst->region_material.size(); ++r)
            if (dst->region_material[r] >= ts->view.n_materials)
                return fail(MCX_ERR_ARG, "region_material[%zu] out of range of the shared materials", r);
        if ((dst->desc.flags & MCX_FLAG_DERIVATIVES) && ts->view.n_materials > MCX_MAX_DMAT)
            return fail(MCX_ERR_ARG, "derivative tallies support at most %d materials", MCX_MAX_DMAT);
    }
    DeviceGuard dg(dst->device);
    if (dst == src) return MCX_OK;
    ts->refs += 1;
    drop_graph(dst);
    release_tables(dst);
    dst->tables = ts;
    if (dst->desc.geometry != MCX_GEOM_NONE)
        TRY(alloc_derivative_tallies(dst, (dst->desc.flags & MCX_FLAG_DERIVATIVES) ? ts->view.n_materials : 0));
    return MCX_OK;
}

int mcx_set_hash_bins(mcx_problem* p, int32_t hash_bins)
{
    g_err.clear();
    TRY(check_tables(p));
    if (hash_bins < 0 || hash_bins > 10000000) return fail(MCX_ERR_ARG, "hash_bins out of range");
    DeviceGuard dg(p->device);
    CUDA_TRY(cudaDeviceSynchronize());
    drop_graph(p);
    return build_hash(p->tables, hash_bins, p->sm_count);
}

int mcx_set_densities(mcx_problem* p, const double* mden, int64_t nnz)
{
    g_err.clear();
    TRY(check_tables(p));
    TableStore* ts = p->tables;
    if (!mden || nnz != ts->nnz) return fail(MCX_ERR_ARG, "expected %lld densities", (long long)ts->nnz);
    for (int64_t i = 0; i < nnz; ++i)
        if (!(mden[i] >= 0.0) || !is_finite(mden[i])) return fail(MCX_ERR_ARG, "mat_dens[%lld] invalid", (long long)i);
    DeviceGuard dg(p->device);
    CUDA_TRY(cudaDeviceSynchronize());
    for (int64_t i = 0; i < nnz; ++i) ts->h_ment[i].w = float_bits((float)mden[i]);
    CUDA_TRY(cudaMemcpy(ts->mden, mden, 8 * nnz, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(ts->ment, ts->h_ment.data(), sizeof(int4) * nnz, cudaMemcpyHostToDevice));
    if (launch_build_pairs(ts->view, ts->tpair, ts->mden2, nnz, p->sm_count * 8, nullptr))
        return fail(MCX_ERR_CUDA, "pair table launch failed");
    CUDA_TRY(cudaDeviceSynchronize());
    return MCX_OK;
}

int mcx_update_tables_device(mcx_problem* p, const double* mat_dens, const double* sigma, void* stream)
{
    g_err.clear();
    TRY(check_tables(p));
    if (!mat_dens && !sigma) return MCX_OK;
    TableStore* ts = p->tables;
    DeviceGuard dg(p->device);
    // the host copy of the entry records no longer reflects device-side densities
    if (mat_dens) ts->h_ment_stale = true;
    if (launch_update_tables(ts->view, mat_dens, mat_dens ? ts->nnz : 0, ts->mden, ts->ment, sigma, ts->sigma,
                             ts->frec, (cudaStream_t)stream))
        return fail(MCX_ERR_CUDA, "table update launch failed");
    // the transport's interval slopes follow the new sigma table, on the same stream
    if (sigma && launch_build_slopes(ts->view, ts->slope, ts->ttot, p->sm_count * 8, (cudaStream_t)stream))
        return fail(MCX_ERR_CUDA, "slope table launch failed");
    if (launch_build_pairs(ts->view, ts->tpair, ts->mden2, ts->nnz, p->sm_count * 8, (cudaStream_t)stream))
        return fail(MCX_ERR_CUDA, "pair table launch failed");
    return MCX_OK;
}

int mcx_set_tuning(mcx_problem* p, const mcx_tune* t)
{
    g_err.clear();
    TRY(check_handle(p));
    if (!t) return fail(MCX_ERR_ARG, "tuning is NULL");
    if (t->mode != MCX_QUEUELESS && t->mode != MCX_QUEUED && t->mode != MCX_QUEUED_FULLEST)
        return fail(MCX_ERR_ARG, "unknown mode");
    if (t->block_size < 32 || t->block_size > 1024 || t->block_size % 32)
        return fail(MCX_ERR_ARG, "block_size must be a multiple of 32 in 32..1024");
    if (t->sort_period < 0) return fail(MCX_ERR_ARG, "sort_period must be >= 0");
    if (t->sort_threshold < 0) return fail(MCX_ERR_ARG, "sort_threshold must be >= 0");
    if (t->iters_per_sync < 1 || t->iters_per_sync > 4096) return fail(MCX_ERR_ARG, "iters_per_sync out of range");
    if (t->max_event_iters < 0) return fail(MCX_ERR_ARG, "max_event_iters must be >= 0");
    if (!(t->time_limit_s >= 0.0)) return fail(MCX_ERR_ARG, "time_limit_s must be >= 0");
    p->tune = *t;
    p->tune.use_graph = t->use_graph ? 1 : 0;
    return MCX_OK;
}

int mcx_run_batch(mcx_problem* p, int64_t first, int64_t n, int64_t pif, uint64_t seed, void* stream)
{
    g_err.clear();
    TRY(check_tables(p));
    if (p->desc.geometry == MCX_GEOM_NONE) return fail(MCX_ERR_STATE, "problem has no geometry");
    if (first < 0 || n < 0 || first + n > p->desc.n_histories)
        return fail(MCX_ERR_ARG, "histories [%lld, %lld) outside [0, %lld)", (long long)first,
                    (long long)(first + n), (long long)p->desc.n_histories);
    DeviceGuard dg(p->device);
    if (n == 0) return MCX_OK;
    mcx_problem* probs[1] = {p};
    return run_loop(p, 1, probs, &first, &n, pif, seed, stream);
}

int mcx_batch_run(int32_t n_problems, mcx_problem* const* problems, const int64_t* n_hist, int64_t pif,
                  uint64_t seed, void* stream)
{
    g_err.clear();
    if (n_problems < 1 || !problems || !n_hist) return fail(MCX_ERR_ARG, "empty problem list");
    TRY(check_tables(problems[0]));
    for (int i = 0; i < n_problems; ++i) {
        TRY(check_handle(problems[i]));
        if (problems[i]->tables != problems[0]->tables)
            return fail(MCX_ERR_ARG, "problem %d does not share problem 0's tables", i);
        if (problems[i]->device != problems[0]->device) return fail(MCX_ERR_ARG, "problem %d on another device", i);
        if (problems[i]->desc.geometry == MCX_GEOM_NONE) return fail(MCX_ERR_ARG, "problem %d has no geometry", i);
        if (problems[i]->M > 0 && n_problems > 1)
            return fail(MCX_ERR_ARG, "problem %d has derivative tallies (single-problem runs only)", i);
        if (n_hist[i] < 0 || n_hist[i] > problems[i]->desc.n_histories)
            return fail(MCX_ERR_ARG, "n_hist[%d] outside [0, n_histories]", i);
        for (int j = 0; j < i; ++j)
            if (problems[j] == problems[i]) return fail(MCX_ERR_ARG, "problem %d listed twice", i);
    }
    DeviceGuard dg(problems[0]->device);
    std::vector<int64_t> first((size_t)n_problems, 0);
    long long total = 0;
    for (int i = 0; i < n_problems; ++i) total += n_hist[i];
    if (total == 0) return MCX_OK;
    return run_loop(problems[0], n_problems, problems, first.data(), n_hist, pif, seed, stream);
}

int mcx_tally_size(const mcx_problem* p, int32_t which, int64_t* n)
{
    g_err.clear();
    TRY(check_handle(p));
    if (!n) return fail(MCX_ERR_ARG, "n is NULL");
    const int64_t B = p->desc.n_batches;
    switch (which) {
    case MCX_TALLY_FLUX:
    case MCX_TALLY_ABSORB: *n = B * p->nb; break;
    case MCX_TALLY_OUTCOME: *n = B * N_OUT; break;
    case MCX_TALLY_DFLUX:
    case MCX_TALLY_DABSORB: *n = B * p->nb * p->M; break;
    case MCX_TALLY_DOUTCOME: *n = B * N_OUT * p->M; break;
    default: return fail(MCX_ERR_ARG, "unknown tally %d", which);
    }
    if (p->desc.geometry == MCX_GEOM_NONE) *n = 0;
    return MCX_OK;
}

int mcx_read_tallies(mcx_problem* p, int32_t which, double* host_out, int64_t n)
{
    g_err.clear();
    int64_t size = 0;
    TRY(mcx_tally_size(p, which, &size));
    if (n != size) return fail(MCX_ERR_ARG, "tally %d has %lld entries, not %lld", which, (long long)size, (long long)n);
    if (n == 0) return MCX_OK;
    if (!host_out) return fail(MCX_ERR_ARG, "host_out is NULL");
    const double* src = which == MCX_TALLY_FLUX ? p->flux
                        : which == MCX_TALLY_ABSORB ? p->absorb
                        : which == MCX_TALLY_OUTCOME ? p->outcome
                        : which == MCX_TALLY_DFLUX ? p->dflux
                        : which == MCX_TALLY_DABSORB ? p->dabsorb
                                                     : p->doutcome;
    DeviceGuard dg(p->device);
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    CUDA_TRY(cudaMemcpy(host_out, src, sizeof(double) * n, cudaMemcpyDeviceToHost));
    return MCX_OK;
}

int mcx_zero_tallies(mcx_problem* p)
{
    g_err.clear();
    TRY(check_handle(p));
    if (p->desc.geometry == MCX_GEOM_NONE) return MCX_OK;
    DeviceGuard dg(p->device);
    // on the problem's own (non-blocking) stream, then wait: the next run on
    // that stream cannot overtake the clearing
    cudaStream_t st = p->stream;
    const int64_t B = p->desc.n_batches;
    CUDA_TRY(cudaMemsetAsync(p->flux, 0, sizeof(double) * B * p->nb, st));
    CUDA_TRY(cudaMemsetAsync(p->absorb, 0, sizeof(double) * B * p->nb, st));
    CUDA_TRY(cudaMemsetAsync(p->outcome, 0, sizeof(double) * B * N_OUT, st));
    if (p->M > 0) {
        CUDA_TRY(cudaMemsetAsync(p->dflux, 0, sizeof(double) * B * p->nb * p->M, st));
        CUDA_TRY(cudaMemsetAsync(p->dabsorb, 0, sizeof(double) * B * p->nb * p->M, st));
        CUDA_TRY(cudaMemsetAsync(p->doutcome, 0, sizeof(double) * B * N_OUT * p->M, st));
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    return MCX_OK;
}

int mcx_read_history_debug(mcx_problem* p, uint32_t* ncoll, int64_t n)
{
    g_err.clear();
    TRY(check_handle(p));
    if (!(p->desc.flags & MCX_FLAG_HISTORY_DEBUG)) return fail(MCX_ERR_STATE, "problem was created without MCX_FLAG_HISTORY_DEBUG");
    if (n < 0 || n > p->debug_n) return fail(MCX_ERR_ARG, "last run had %lld histories", (long long)p->debug_n);
    if (n == 0) return MCX_OK;
    if (!ncoll) return fail(MCX_ERR_ARG, "ncoll is NULL");
    DeviceGuard dg(p->device);
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    CUDA_TRY(cudaMemcpy(ncoll, p->ncoll_debug, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost));
    return MCX_OK;
}

int mcx_set_kernel_timing(mcx_problem* p, int32_t on)
{
    g_err.clear();
    TRY(check_handle(p));
    if (on != 0 && on != 1) return fail(MCX_ERR_ARG, "on must be 0 or 1");
    p->kernel_timing = on;
    return MCX_OK;
}

int mcx_last_kernel_stats(const mcx_problem* p, double* ms, int64_t* counts)
{
    g_err.clear();
    TRY(check_handle(p));
    if (!ms || !counts) return fail(MCX_ERR_ARG, "NULL buffer");
    for (int e = 0; e < 3; ++e) ms[e] = p->kernel_timing ? p->kt_ms[e] : -1.0;
    for (int e = 0; e < 4; ++e) counts[e] = p->kt_count[e];
    return MCX_OK;
}

int mcx_last_run_stats(const mcx_problem* p, int64_t* out, int32_t n)
{
    g_err.clear();
    TRY(check_handle(p));
    if (!out || n < 3) return fail(MCX_ERR_ARG, "need room for 3 values");
    for (int i = 0; i < 3; ++i) out[i] = p->stats[i];
    for (int i = 3; i < n && i < 6; ++i) out[i] = p->stats[i];
    return MCX_OK;
}

int mcx_xs_lookup(mcx_problem* p, int64_t n, const double* E, const int32_t* mat, void* out,
                  int32_t flags, void* stream)
{
    g_err.clear();
    TRY(check_tables(p));
    if (n < 0) return fail(MCX_ERR_ARG, "n must be >= 0");
    if (n >= ((int64_t)1 << 31)) return fail(MCX_ERR_ARG, "n must be < 2^31");
    if (flags & ~(MCX_LOOKUP_FAST | MCX_LOOKUP_SORT | MCX_LOOKUP_STAGED | MCX_LOOKUP_OUT32 | MCX_LOOKUP_LINEAR))
        return fail(MCX_ERR_ARG, "unknown lookup flags");
    if ((flags & (MCX_LOOKUP_OUT32 | MCX_LOOKUP_LINEAR)) && !(flags & MCX_LOOKUP_FAST))
        return fail(MCX_ERR_ARG, "MCX_LOOKUP_OUT32 and MCX_LOOKUP_LINEAR need MCX_LOOKUP_FAST");
    if (n == 0) return MCX_OK;
    if (!E || !mat || !out) return fail(MCX_ERR_ARG, "NULL buffer");
    DeviceGuard dg(p->device);
    return lookup_device(p, n, E, mat, out, flags, (cudaStream_t)stream);
}

int mcx_xs_sort(mcx_problem* p, int64_t n, const double* E, const int32_t* mat, int32_t* perm,
                void* stream)
{
    g_err.clear();
    TRY(check_tables(p));
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(MCX_ERR_ARG, "n out of range");
    if (n == 0) return MCX_OK;
    if (!E || !mat || !perm) return fail(MCX_ERR_ARG, "NULL buffer");
    DeviceGuard dg(p->device);
    return sort_device(p, n, E, mat, perm, (cudaStream_t)stream);
}

int mcx_xs_sort_inputs(mcx_problem* p, int64_t n, const double* E, const int32_t* mat, int32_t* perm,
                       double* E_binned, int32_t* mat_binned, void* stream)
{
    g_err.clear();
    TRY(check_tables(p));
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(MCX_ERR_ARG, "n out of range");
    if (n == 0) return MCX_OK;
    if (!E || !mat || !perm || !E_binned || !mat_binned) return fail(MCX_ERR_ARG, "NULL buffer");
    DeviceGuard dg(p->device);
    return sort_device(p, n, E, mat, perm, (cudaStream_t)stream, kLookupsPerBucket, E_binned, mat_binned);
}

int mcx_xs_lookup_ordered(mcx_problem* p, int64_t n, const double* E, const int32_t* mat,
                          const int32_t* perm, void* out, int32_t flags, void* stream)
{
    g_err.clear();
    TRY(check_tables(p));
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(MCX_ERR_ARG, "n out of range");
    if (flags & ~(MCX_LOOKUP_FAST | MCX_LOOKUP_STAGED | MCX_LOOKUP_OUT32 | MCX_LOOKUP_LINEAR |
                  MCX_LOOKUP_BINNED_INPUTS))
        return fail(MCX_ERR_ARG, "flags may hold MCX_LOOKUP_FAST, MCX_LOOKUP_STAGED, MCX_LOOKUP_OUT32, "
                                 "MCX_LOOKUP_LINEAR and MCX_LOOKUP_BINNED_INPUTS only");
    if ((flags & (MCX_LOOKUP_OUT32 | MCX_LOOKUP_LINEAR)) && !(flags & MCX_LOOKUP_FAST))
        return fail(MCX_ERR_ARG, "MCX_LOOKUP_OUT32 and MCX_LOOKUP_LINEAR need MCX_LOOKUP_FAST");
    if ((flags & MCX_LOOKUP_BINNED_INPUTS) &&
        (!(flags & MCX_LOOKUP_FAST) || (flags & MCX_LOOKUP_STAGED) || !perm))
        return fail(MCX_ERR_ARG, "MCX_LOOKUP_BINNED_INPUTS needs MCX_LOOKUP_FAST, a permutation and no "
                                 "MCX_LOOKUP_STAGED");
    if (n == 0) return MCX_OK;
    if (!E || !mat || !out) return fail(MCX_ERR_ARG, "NULL buffer");
    DeviceGuard dg(p->device);
    return lookup_device_ordered(p, n, E, mat, perm, out, flags, (cudaStream_t)stream);
}

int mcx_xs_lookup_host(mcx_problem* p, int64_t n, const double* E_host, const int32_t* mat_host,
                       void* out_host, int32_t flags)
{
    g_err.clear();
    TRY(check_tables(p));
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(MCX_ERR_ARG, "n out of range");
    if (flags & ~(MCX_LOOKUP_FAST | MCX_LOOKUP_SORT | MCX_LOOKUP_STAGED | MCX_LOOKUP_OUT32 | MCX_LOOKUP_LINEAR))
        return fail(MCX_ERR_ARG, "unknown lookup flags");
    if ((flags & (MCX_LOOKUP_OUT32 | MCX_LOOKUP_LINEAR)) && !(flags & MCX_LOOKUP_FAST))
        return fail(MCX_ERR_ARG, "MCX_LOOKUP_OUT32 and MCX_LOOKUP_LINEAR need MCX_LOOKUP_FAST");
    if (n == 0) return MCX_OK;
    if (!E_host || !mat_host || !out_host) return fail(MCX_ERR_ARG, "NULL buffer");
    const size_t es = (flags & MCX_LOOKUP_OUT32) ? sizeof(float) : sizeof(double);
    DeviceGuard dg(p->device);
    const TableStore* ts = p->tables;
    const int nc = ts->view.n_ch;
    const int64_t most = (flags & MCX_LOOKUP_OUT32) ? kHostChunk32 : kHostChunk;
    const int64_t chunk = n < most ? n : most;
    const SortParams sp = batch_sort_params(ts, chunk);
    const int64_t nbins = (int64_t)sp.n_materials * sp.n_ebuckets + 1 + kSortScanParts;
    // staging per slot (in doubles): E [chunk], mat [chunk int32], out
    // [chunk * nc], binning permutation [chunk int32], bin scratch [nbins
    // uint32, rounded up to whole doubles]
    const int64_t per = chunk * (4 + nc) + (nbins + 1) / 2;
    if (p->h_buf_cap < kHostSlots * per) {
        dev_free(p->h_buf);
        p->h_buf_cap = 0;
        TRY(dev_alloc(&p->h_buf, (size_t)(kHostSlots * per)));
        p->h_buf_cap = kHostSlots * per;
    }
    for (cudaStream_t& hs : p->hstream)
        if (!hs) CUDA_TRY(cudaStreamCreateWithFlags(&hs, cudaStreamNonBlocking));
    cudaStream_t ss[4] = {p->stream, p->stream2, p->hstream[0], p->hstream[1]};
    for (int64_t off = 0, c = 0; off < n; off += chunk, ++c) {
        const int64_t m = n - off < chunk ? n - off : chunk;
        const int slot = (int)(c % kHostSlots);
        cudaStream_t st = ss[slot];
        double* base = p->h_buf + slot * per;
        double* dE = base;
        int32_t* dM = (int32_t*)(base + chunk);
        double* dO = base + 2 * chunk;
        int32_t* dP = (int32_t*)(base + chunk * (2 + nc));
        uint32_t* dB = (uint32_t*)(base + chunk * (3 + nc));
        CUDA_TRY(cudaMemcpyAsync(dE, E_host + off, 8 * m, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(dM, mat_host + off, 4 * m, cudaMemcpyHostToDevice, st));
        const int32_t* perm = nullptr;
        if (flags & MCX_LOOKUP_SORT) {
            if (launch_lookup_sort(sp, m, dE, dM, dB, dP, lookup_grid(p), st))
                return fail(MCX_ERR_CUDA, "lookup sort launch failed");
            perm = dP;
        }
        TRY(lookup_device_ordered(p, m, dE, dM, perm, dO,
                                  flags & (MCX_LOOKUP_FAST | MCX_LOOKUP_STAGED | MCX_LOOKUP_OUT32 | MCX_LOOKUP_LINEAR), st, slot));
        CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(out_host) + (size_t)off * nc * es, dO, es * m * nc,
                                 cudaMemcpyDeviceToHost, st));
    }
    for (int k = 0; k < kHostSlots; ++k) CUDA_TRY(cudaStreamSynchronize(ss[k]));
    if (flags & MCX_LOOKUP_STAGED) return mcx_check_device(p, nullptr);
    return MCX_OK;
}

int mcx_xs_indices(mcx_problem* p, int64_t n, const double* E, const int32_t* mat, int32_t max_species,
                   int32_t* kout, void* stream)
{
    g_err.clear();
    TRY(check_tables(p));
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(MCX_ERR_ARG, "n out of range");
    if (max_species < p->tables->view.max_mat_species)
        return fail(MCX_ERR_ARG, "max_species must be >= %d", p->tables->view.max_mat_species);
    if (n == 0) return MCX_OK;
    if (!E || !mat || !kout) return fail(MCX_ERR_ARG, "NULL buffer");
    DeviceGuard dg(p->device);
    if (launch_xs_indices(p->tables->view, n, E, mat, max_species, kout, lookup_grid(p), (cudaStream_t)stream))
        return fail(MCX_ERR_CUDA, "index kernel launch failed");
    return MCX_OK;
}

int mcx_xs_lookup_backward(mcx_problem* p, int64_t n, const double* E, const int32_t* mat,
                           const double* grad_out, double* grad_dens, double* grad_sigma, void* stream)
{
    g_err.clear();
    TRY(check_tables(p));
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(MCX_ERR_ARG, "n out of range");
    if (n == 0) return MCX_OK;
    if (!E || !mat || !grad_out || !grad_dens || !grad_sigma) return fail(MCX_ERR_ARG, "NULL buffer");
    DeviceGuard dg(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    // binned order, then warps that aggregate per species and grid interval
    TRY(ensure_lookup_scratch(p, n, 0));
    TRY(sort_device(p, n, E, mat, p->perm, st, kBackwardLookupsPerBucket));
    TRY(ensure_work_ctr(p));
    if (launch_xs_backward_binned(p->tables->view, p->tables->nnz, n, E, mat, p->perm, grad_out, grad_dens,
                                  grad_sigma, p->sm_count, p->work_ctr, st))
        return fail(MCX_ERR_CUDA, "backward kernel launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return MCX_OK;
}

int mcx_debug_uniforms(uint64_t seed, uint32_t problem_id, uint64_t hist, uint32_t first, int64_t n,
                       double* out, void* stream)
{
    g_err.clear();
    if (n < 0) return fail(MCX_ERR_ARG, "n must be >= 0");
    if (n == 0) return MCX_OK;
    if (!out) return fail(MCX_ERR_ARG, "out is NULL");
    if (launch_debug_uniforms(rng_key(seed, problem_id), hist, first, n, out, (cudaStream_t)stream))
        return fail(MCX_ERR_CUDA, "uniforms kernel launch failed");
    return MCX_OK;
}

int mcx_debug_transport_xs(mcx_problem* p, int64_t n, const double* E, const int32_t* mat, double* out,
                           void* stream)
{
    g_err.clear();
    TRY(check_tables(p));
    if (n < 0 || n > ((int64_t)1 << 24)) return fail(MCX_ERR_ARG, "n must be in [0, 2^24]");
    if (n == 0) return MCX_OK;
    if (!E || !mat || !out) return fail(MCX_ERR_ARG, "NULL buffer");
    const int nc = p->tables->view.n_ch;
    if (nc != 2 && nc != 3 && nc != 5) return fail(MCX_ERR_ARG, "transport needs 2, 3 or 5 channels");
    DeviceGuard dg(p->device);
    // running sums, 8 bytes each, rows of a multiple of 4 entries as the lookup stores them
    const int64_t stride = ((p->tables->view.max_mat_species > 0 ? p->tables->view.max_mat_species : 1) + 3) & ~(int64_t)3;
    double* scratch = nullptr;
    TRY(dev_alloc(&scratch, (size_t)(n * stride)));
    cudaStream_t st = (cudaStream_t)stream;
    const int rc = launch_debug_transport_xs(p->tables->view, n, E, mat, reinterpret_cast<float2*>(scratch), stride,
                                             out, st);
    const cudaError_t es = cudaStreamSynchronize(st);
    dev_free(scratch);
    if (rc || es != cudaSuccess) return fail(MCX_ERR_CUDA, "transport lookup kernel failed");
    return MCX_OK;
}

int mcx_debug_neg_log(const double* x, int64_t n, double* out, void* stream)
{
    g_err.clear();
    if (n < 0) return fail(MCX_ERR_ARG, "n must be >= 0");
    if (n == 0) return MCX_OK;
    if (!x || !out) return fail(MCX_ERR_ARG, "NULL buffer");
    if (launch_debug_neg_log(x, n, out, (cudaStream_t)stream))
        return fail(MCX_ERR_CUDA, "logarithm kernel launch failed");
    return MCX_OK;
}

int mcx_run_eigenvalue(mcx_problem* p, int64_t n_per_gen, int32_t n_generations, int32_t n_inactive,
                       double k0, double T_fission, int64_t particles_in_flight, uint64_t seed,
                       double* gen_out, void* stream)
{
    g_err.clear();
    TRY(check_tables(p));
    if (p->desc.geometry == MCX_GEOM_NONE) return fail(MCX_ERR_STATE, "problem has no geometry");
    if (p->tables->view.ch_nu_fission < 0)
        return fail(MCX_ERR_ARG, "an eigenvalue run needs a nu-fission channel (3- or 5-channel tables)");
    if (n_per_gen < 1 || n_per_gen > INT32_MAX) return fail(MCX_ERR_ARG, "n_per_gen out of range");
    if (n_generations < 1 || n_inactive < 0 || n_inactive >= n_generations)
        return fail(MCX_ERR_ARG, "need 0 <= n_inactive < n_generations");
    if (!(k0 > 0.0) || !is_finite(k0)) return fail(MCX_ERR_ARG, "k0 must be positive and finite");
    if (!(T_fission > 0.0) || !is_finite(T_fission)) return fail(MCX_ERR_ARG, "T_fission must be positive");
    if (!gen_out) return fail(MCX_ERR_ARG, "gen_out is NULL");
    if (p->M > 0) return fail(MCX_ERR_ARG, "derivative tallies are not supported in eigenvalue runs");
    if ((double)n_generations * (double)n_per_gen > 9.0e18) return fail(MCX_ERR_ARG, "too many histories");
    DeviceGuard dg(p->device);
    const int64_t N = n_per_gen;
    const int64_t n_active = n_generations - n_inactive;
    TRY(ensure_eigen(p, N, std::max<int64_t>(4 * N, 4096)));
    cudaStream_t st = p->stream;
    const int grid = p->sm_count * 8;
    double k_norm = k0;
    mcx_problem* probs[1] = {p};
    for (int32_t g = 0; g < n_generations; ++g) {
        const bool active = g >= n_inactive;
        if (g == n_inactive) TRY(mcx_zero_tallies(p));
        EigenCtl h{};
        for (int attempt = 0;; ++attempt) {
            CUDA_TRY(cudaMemsetAsync(p->e_ctl, 0, sizeof(EigenCtl), st));
            CUDA_TRY(cudaMemsetAsync(p->e_count, 0, sizeof(uint32_t) * N, st));
            EigenGen eg;
            eg.tally_off = active ? (int64_t)n_inactive * N : (int64_t)g * N;
            eg.n_hist_total = active ? n_active * N : N;
            eg.src = g > 0 ? p->e_src : nullptr;
            eg.k_norm = k_norm;
            eg.T_fission = T_fission;
            eg.bank = p->e_bank;
            eg.bank_key = p->e_key;
            eg.bank_cap = p->e_bank_cap;
            eg.site_count = p->e_count;
            eg.eig = p->e_ctl;
            const int64_t first = (int64_t)g * N, count = N;
            // the generation's histories run on the problem's stream after
            // the memsets above (run_loop orders the user stream before it)
            CUDA_TRY(cudaStreamSynchronize(st));
            TRY(run_loop(p, 1, probs, &first, &count, particles_in_flight, seed, stream, &eg));
            CUDA_TRY(cudaMemcpyAsync(&h, p->e_ctl, sizeof(EigenCtl), cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            if (h.banked <= (unsigned long long)p->e_bank_cap) break;
            // the bank overflowed: the generation's histories are fixed by
            // their keys, so an inactive generation is simply run again with
            // room for every site; an active one has already scored
            if (active || attempt >= 2)
                return fail(MCX_ERR_BOUNDS, "fission bank overflow in generation %d: %llu sites, capacity %lld",
                            g, h.banked, (long long)p->e_bank_cap);
            const int64_t need = (int64_t)h.banked + (int64_t)(h.banked / 4) + 1024;
            if (need > ((int64_t)1 << 31)) return fail(MCX_ERR_BOUNDS, "fission bank of %llu sites is too large", h.banked);
            TRY(ensure_eigen(p, N, need));
        }
        const int64_t M = (int64_t)h.banked;
        const double k_g = ((double)M * k_norm) / (double)N;
        gen_out[4 * g + 0] = k_g;
        gen_out[4 * g + 1] = h.k_col / (double)N;
        gen_out[4 * g + 2] = h.k_tl / (double)N;
        gen_out[4 * g + 3] = (double)M;
        if (M == 0) {
            p->e_last_M = 0;
            return fail(MCX_ERR_STATE, "generation %d banked no fission site", g);
        }
        // canonical order (parent history, sequence), then the next source
        unsigned long long total = 0ull, bad = 0ull;
        if (launch_site_offsets(p->e_count, N, p->e_tiles, p->e_off, st))
            return fail(MCX_ERR_CUDA, "site offset kernels failed to launch");
        CUDA_TRY(cudaMemsetAsync(p->e_bad, 0, sizeof(unsigned long long), st));
        if (launch_bank_order(p->e_bank, p->e_key, M, p->e_off, N, M, p->e_ordered, p->e_bad, grid, st))
            return fail(MCX_ERR_CUDA, "bank order kernel failed to launch");
        CUDA_TRY(cudaMemcpyAsync(&total, p->e_tiles + bank_scan_tiles(N), sizeof(total), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaMemcpyAsync(&bad, p->e_bad, sizeof(bad), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        if (total != (unsigned long long)M || bad != 0ull)
            return fail(MCX_ERR_STATE, "generation %d: %llu sites banked, %llu counted by histories, %llu misplaced",
                        g, (unsigned long long)M, total, bad);
        p->e_last_M = M;
        if (g + 1 < n_generations) {
            if (launch_bank_resample(p->e_ordered, M, N, p->e_src, grid, st))
                return fail(MCX_ERR_CUDA, "resample kernel failed to launch");
        }
        k_norm = k_g;
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    return MCX_OK;
}

int mcx_check_device(mcx_problem* p, void* stream)
{
    g_err.clear();
    TRY(check_handle(p));
    DeviceGuard dg(p->device);
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    if (MCX_BOUNDS_CHECK) {
        // every kernel translation unit's first failed check (each word is
        // cleared by its read)
        const unsigned long long e[4] = {bounds_error_xs_exact(), bounds_error_xs_fast(), bounds_error_adjoint(),
                                         bounds_error_transport()};
        const char* unit[4] = {"exact lookup", "fast lookup", "adjoint", "transport"};
        for (int i = 0; i < 4; ++i)
            if (e[i]) return bounds_failure(e[i], unit[i]);
    }
    if (!p->work_ctr) return MCX_OK;
    unsigned long long w = 0ull;
    CUDA_TRY(cudaMemcpy(&w, p->work_ctr + kWorkCtrs, sizeof(w), cudaMemcpyDeviceToHost));
    if (w == 0ull) return MCX_OK;
    CUDA_TRY(cudaMemset(p->work_ctr + kWorkCtrs, 0, sizeof(w)));
    return fail(MCX_ERR_TIMEOUT, "a staged lookup kernel gave up waiting on its pipeline");
}

int mcx_bounds_checked(void) { return MCX_BOUNDS_CHECK; }

int mcx_fission_bank_size(const mcx_problem* p, int64_t* n)
{
    g_err.clear();
    TRY(check_handle(p));
    if (!n) return fail(MCX_ERR_ARG, "n is NULL");
    *n = p->e_last_M;
    return MCX_OK;
}

int mcx_read_fission_bank(mcx_problem* p, double* rows, int64_t n)
{
    g_err.clear();
    TRY(check_handle(p));
    if (n < 0 || n > p->e_last_M) return fail(MCX_ERR_ARG, "n must be in [0, %lld]", (long long)p->e_last_M);
    if (n == 0) return MCX_OK;
    if (!rows) return fail(MCX_ERR_ARG, "rows is NULL");
    DeviceGuard dg(p->device);
    std::vector<FissionSite> h((size_t)n);
    CUDA_TRY(cudaMemcpyAsync(h.data(), p->e_ordered, sizeof(FissionSite) * n, cudaMemcpyDeviceToHost, p->stream));
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    const int32_t ln = p->desc.geometry == MCX_GEOM_LATTICE && p->desc.lattice_n > 0 ? p->desc.lattice_n : 1;
    for (int64_t i = 0; i < n; ++i) {
        double* r = rows + 6 * i;
        r[0] = h[i].x;
        r[1] = h[i].y;
        r[2] = h[i].z;
        r[3] = (double)(h[i].cell / ln);
        r[4] = (double)(h[i].cell % ln);
        r[5] = (double)h[i].inpin;
    }
    return MCX_OK;
}

}  // extern "C"
