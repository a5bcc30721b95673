// eigen.cu -- fission bank of an eigenvalue generation: put the banked sites
// in a canonical order and resample them into the next generation's source.
//
// The event kernels bank sites in whatever order the GPU reaches them, each
// with its key (history of the run, sequence number within that history) and
// every history records how many sites it banked.  Ordering by key is then a
// placement, not a sort: offset[h] = exclusive prefix sum of the per-history
// counts, site (h, q) goes to offset[h] + q.  That is the order a sequential
// run of the histories would bank them in, so the next generation does not
// depend on the GPU's scheduling.  The next source is the systematic
// resample source[i] = bank[floor(i M / N)] of the M ordered sites.
#include "kernels.h"

namespace mcx {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kTile = kScanThreads * kScanItems;
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ unsigned long long warp_incl_scan(unsigned long long v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Exclusive block scan of one value per thread (blockDim.x == kScanThreads);
// *total receives the block's sum.
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v,
                                                              unsigned long long* total)
{
    __shared__ unsigned long long warp_tot[kScanThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned long long incl = warp_incl_scan(v);
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const unsigned long long t = warp_incl_scan(warp_tot[lane]);
        warp_tot[lane] = t;
    }
    __syncthreads();
    const unsigned long long before = wid ? warp_tot[wid - 1] : 0ull;
    *total = warp_tot[kScanThreads / 32 - 1];
    __syncthreads();
    return before + incl - v;
}

__global__ void __launch_bounds__(kScanThreads) k_tile_sums(const uint32_t* __restrict__ cnt, int64_t n,
                                                            unsigned long long* __restrict__ tile_sum)
{
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kScanItems;
    unsigned long long s = 0ull;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += cnt[base + k];
    unsigned long long total;
    block_excl_scan(s, &total);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

// In-place exclusive scan of the tile sums (one block); tile_sum[n_tiles]
// receives the grand total.
__global__ void __launch_bounds__(kScanThreads) k_scan_tile_sums(unsigned long long* tile_sum, int64_t n_tiles)
{
    unsigned long long carry = 0ull;
    for (int64_t base = 0; base < n_tiles; base += kScanThreads) {
        const int64_t i = base + threadIdx.x;
        const unsigned long long v = i < n_tiles ? tile_sum[i] : 0ull;
        unsigned long long total;
        const unsigned long long ex = block_excl_scan(v, &total);
        if (i < n_tiles) tile_sum[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) tile_sum[n_tiles] = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_tile_offsets(const uint32_t* __restrict__ cnt, int64_t n,
                                                               const unsigned long long* __restrict__ tile_pref,
                                                               unsigned long long* __restrict__ off)
{
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    unsigned long long s = 0ull;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? cnt[base + k] : 0u;
        s += v[k];
    }
    unsigned long long total;
    unsigned long long run = tile_pref[blockIdx.x] + block_excl_scan(s, &total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) off[base + k] = run;
        run += v[k];
    }
}

// Site j of the staging bank goes to offset[history] + sequence.  A key that
// points outside [0, M) (an inconsistent bank) is counted, not written.
__global__ void k_bank_order(const FissionSite* __restrict__ bank, const int2* __restrict__ key, int64_t n_banked,
                             const unsigned long long* __restrict__ off, int64_t n_hist, int64_t M,
                             FissionSite* __restrict__ ordered, unsigned long long* __restrict__ bad)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_banked;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int2 k = key[j];
        const bool ok_h = k.x >= 0 && (int64_t)k.x < n_hist && k.y >= 0;
        const unsigned long long dst = ok_h ? off[k.x] + (unsigned long long)k.y : ~0ull;
        if (ok_h && dst < (unsigned long long)M) ordered[dst] = bank[j];
        else atomicAdd(bad, 1ull);
    }
}

__global__ void k_bank_resample(const FissionSite* __restrict__ ordered, int64_t M, int64_t N,
                                FissionSite* __restrict__ src)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        src[i] = ordered[(int64_t)(((unsigned long long)i * (unsigned long long)M) / (unsigned long long)N)];
}

}  // namespace

int64_t bank_scan_tiles(int64_t n) { return (n + kTile - 1) / kTile; }

int launch_site_offsets(const uint32_t* cnt, int64_t n, unsigned long long* tile_sum,
                        unsigned long long* off, cudaStream_t st)
{
    const int64_t tiles = bank_scan_tiles(n);
    if (tiles < 1 || tiles > INT32_MAX) return -1;
    k_tile_sums<<<(unsigned)tiles, kScanThreads, 0, st>>>(cnt, n, tile_sum);
    k_scan_tile_sums<<<1, kScanThreads, 0, st>>>(tile_sum, tiles);
    k_tile_offsets<<<(unsigned)tiles, kScanThreads, 0, st>>>(cnt, n, tile_sum, off);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_bank_order(const FissionSite* bank, const int2* key, int64_t n_banked,
                      const unsigned long long* off, int64_t n_hist, int64_t M, FissionSite* ordered,
                      unsigned long long* bad, int grid, cudaStream_t st)
{
    if (n_banked > 0) k_bank_order<<<grid, 256, 0, st>>>(bank, key, n_banked, off, n_hist, M, ordered, bad);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_bank_resample(const FissionSite* ordered, int64_t M, int64_t N, FissionSite* src, int grid,
                         cudaStream_t st)
{
    if (M < 1 || N < 1) return -1;
    k_bank_resample<<<grid, 256, 0, st>>>(ordered, M, N, src);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace mcx
