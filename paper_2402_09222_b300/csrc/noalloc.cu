// noalloc.cu -- the binned macroscopic lookup for callers that cannot
// allocate device memory.
//
// mcx_xs_lookup with MCX_LOOKUP_SORT allocates its scratch (the binning
// permutation and the bin counters) with cudaMalloc on first use.  Some
// callers cannot let a library do that: processes whose device memory is
// fully reserved up front by another allocator (a framework's memory pool
// or a fixed per-process budget) and for which an extra driver allocation
// would fail or break the budget, and latency-bound loops for which
// cudaMalloc's implicit device synchronisation and unbounded latency are
// not acceptable.  For them, mcx_xs_lookup_binned_static does the same work
// with its scratch in file-scope device arrays of fixed size, created when
// the library is loaded onto a device and held by that device until the
// process exits (about 4.05 MB per device).  The arrays' device addresses
// are looked up once per device and kept for the life of the process, so
// the entry point must not be used on a device after cudaDeviceReset (or
// any other teardown of its primary context) in the same process.
#include <mutex>

#include "kernels.h"

namespace {

// Scratch shared by every call of the entry point on a device.
static __device__ __align__(256) int32_t g_static_perm[MCX_STATIC_MAX_LOOKUPS];
static __device__ __align__(256) uint32_t g_static_bins[MCX_STATIC_MAX_BINS + 1 + mcx::kSortScanParts];
// Chunk counter of the fast lookup's in-order sweep of the binned order
// (zeroed on the stream by every launch).
static __device__ __align__(256) unsigned long long g_static_work;

constexpr int kMaxDevices = 64;

struct ScratchAddr {
    bool ready = false;
    int32_t* perm = nullptr;
    uint32_t* bins = nullptr;
    unsigned long long* work = nullptr;
};

ScratchAddr g_addr[kMaxDevices];
std::mutex g_mu;

// Device addresses of the scratch arrays on `dev` (which must be current).
// In host code the arrays' names only stand in for them, so the addresses
// are looked up once per device with cudaGetSymbolAddress.
int scratch_on(int dev, ScratchAddr* out)
{
    if (dev < 0 || dev >= kMaxDevices)
        return mcx::set_error(MCX_ERR_ARG, "device ordinal beyond the static-scratch table");
    std::lock_guard<std::mutex> lock(g_mu);
    ScratchAddr& a = g_addr[dev];
    if (!a.ready) {
        void* pp = nullptr;
        void* pb = nullptr;
        cudaError_t e1 = cudaGetSymbolAddress(&pp, g_static_perm);
        if (e1 != cudaSuccess)
            return mcx::set_error(MCX_ERR_CUDA, cudaGetErrorString(e1));
        cudaError_t e2 = cudaGetSymbolAddress(&pb, g_static_bins);
        if (e2 != cudaSuccess)
            return mcx::set_error(MCX_ERR_CUDA, cudaGetErrorString(e2));
        void* pw = nullptr;
        cudaError_t e3 = cudaGetSymbolAddress(&pw, g_static_work);
        if (e3 != cudaSuccess)
            return mcx::set_error(MCX_ERR_CUDA, cudaGetErrorString(e3));
        a.perm = static_cast<int32_t*>(pp);
        a.bins = static_cast<uint32_t*>(pb);
        a.work = static_cast<unsigned long long*>(pw);
        a.ready = true;
    }
    *out = a;
    return MCX_OK;
}

}  // namespace

extern "C" int mcx_xs_lookup_binned_static(mcx_problem* p, int64_t n, const double* E,
                                           const int32_t* mat, double* out, int32_t flags,
                                           void* stream)
{
    mcx::LookupView v;
    int rc = mcx::problem_lookup_view(p, &v);
    if (rc != MCX_OK) return rc;
    if (n < 0) return mcx::set_error(MCX_ERR_ARG, "n must be >= 0");
    if (n > MCX_STATIC_MAX_LOOKUPS)
        return mcx::set_error(MCX_ERR_ARG,
                              "n exceeds MCX_STATIC_MAX_LOOKUPS (1048576) of the static-scratch lookup; "
                              "split the batch or use mcx_xs_lookup");
    if (flags & ~MCX_LOOKUP_FAST) return mcx::set_error(MCX_ERR_ARG, "flags may hold MCX_LOOKUP_FAST only");
    const mcx::SortParams sp = mcx::lookup_sort_params(v.sort.n_materials, v.emin, v.emax, n, MCX_STATIC_MAX_BINS);
    const int64_t nbins = (int64_t)sp.n_materials * sp.n_ebuckets;
    if (nbins > MCX_STATIC_MAX_BINS)
        return mcx::set_error(MCX_ERR_ARG, "too many materials for the static bin array");
    if (n == 0) return MCX_OK;
    if (!E || !mat || !out) return mcx::set_error(MCX_ERR_ARG, "NULL buffer");
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != v.device && cudaSetDevice(v.device) != cudaSuccess)
        return mcx::set_error(MCX_ERR_CUDA, "cudaSetDevice failed");
    ScratchAddr a;
    rc = scratch_on(v.device, &a);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (rc == MCX_OK) {
        // the bin counters are cleared inside launch_lookup_sort and the chunk
        // counter inside launch_xs_lookup_fast (they keep the previous call's
        // contents otherwise); the permutation is fully rewritten.  The fast
        // form sweeps the binned order front to back with chunk-claiming
        // warps on one resident grid, as the allocating binned lookup does.
        if (mcx::launch_lookup_sort(sp, n, E, mat, a.bins, a.perm, v.grid, st))
            rc = mcx::set_error(MCX_ERR_CUDA, "binning launch failed");
        else if ((flags & MCX_LOOKUP_FAST)
                     ? mcx::launch_xs_lookup_fast(v.tables, n, E, mat, a.perm, out, false,
                                                  v.sm_count * mcx::kFastBlocksPerSm, st, a.work)
                     : mcx::launch_xs_lookup_exact(v.tables, n, E, mat, a.perm, out, v.grid, st))
            rc = mcx::set_error(MCX_ERR_CUDA, "lookup launch failed");
    }
    if (prev >= 0 && prev != v.device) cudaSetDevice(prev);
    return rc;
}
