// xs_fast.cu -- macroscopic lookup with FP32 interpolation weights and
// compensated FP32 sums, and the binning of lookups by material and energy.
//
// B300 runs FP64 at 1/64 of its FP32 rate, so the FP64 work of the plain
// definition (a division and ~5 multiply-adds per channel and species) makes
// the exact lookup FP64-bound long before HBM is.  Here the grid search stays
// exact (integer compares of FP64 bit patterns) and no FP64 operation is left
// in the per-species loop:
//   E - g[k] = (E_hi - g_hi) + (E_lo - g_lo)     with (hi, lo) FP32 pairs
// where x_hi = float(x), x_lo = float(x - x_hi) (stored for the grid, formed
// once per lookup for E).  For neighbouring energies E_hi - g_hi is exact
// (Sterbenz) and the lo parts carry the remaining ~2^-24 of the value, so the
// distance keeps a relative error of about 2^-23; then
//   w1 = (E - g[k]) / (g[k+1] - g[k]),  w0 = (g[k+1] - E) / (g[k+1] - g[k])
//   sigma = w0 * s[k] + w1 * s[k+1]          (both terms >= 0: no cancellation)
//   Sigma_r accumulated as an unevaluated FP32 pair (hi, lo) with TwoSum.
// Error budget (u = 2^-24): the distances a, b carry ~2u, a + b one more,
// the fast division 2 ulp and the two weight products one each, so a weight
// is within ~6u; the U species' 2U weighted terms of a group are added with
// fused multiply-adds (2U roundings, 8u at U = 4) and the groups are
// accumulated compensated (~1u).  All terms are non-negative, so the errors
// do not amplify: each output is within ~15u = 9e-7 of the FP64 definition,
// under the 1e-6 bound (the largest measured on 1e6 samples: 3.7e-7).
#include "kernels.h"

namespace mcx {

namespace {

// Species in flight per thread and minimum resident 256-thread blocks per SM
// (the register cap that follows); 4 and 4 measured fastest on B300 among
// U in {1, 2, 4} x blocks in {1, 4, 5}.
#ifndef MCX_FAST_UNROLL
#define MCX_FAST_UNROLL 4
#endif
#ifndef MCX_FAST_MIN_BLOCKS
#define MCX_FAST_MIN_BLOCKS 4
#endif
// Fast division for the density-scaled weight (<= 2 ulp): measured 9 % faster
// than an IEEE-rounded reciprocal and still inside the 1e-6 budget.
#ifndef MCX_FAST_FDIV
#define MCX_FAST_FDIV 1
#endif
// Per channel, add both weighted table values with two fused multiply-adds
// (instead of a multiply, a fused multiply-add and an add): 3 % faster.
#ifndef MCX_FAST_FMA2
#define MCX_FAST_FMA2 1
#endif
// Streaming (evict-first) loads of the per-lookup inputs and stores of the
// outputs, so that they do not displace table records from L1: 2 % faster.
#ifndef MCX_FAST_STREAM
#define MCX_FAST_STREAM 1
#endif
// Skip the search probe (and its dependent load) when the candidate range has
// already shrunk to one point -- the common case with a fine hash grid (at
// 68400 bins 83 % of the windows hold one point): in natural order 306 ->
// 221 ms per 1e8 lookups (one DRAM sector less per species), binned 1 %.
#ifndef MCX_FAST_SKIP
#define MCX_FAST_SKIP 1
#endif
constexpr int kFastUnroll = MCX_FAST_UNROLL;
constexpr int kSmemBins = 12288;   // histograms up to this size count in shared memory
constexpr int kChunk = 128;        // lookups a warp claims at a time in binned order

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x)
{
    const float s = hi + x;
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += e;
}

// One thread per lookup; the material's species are taken U at a time so
// that the U independent chains of loads (window, search probes, point
// records) overlap.  The search inside a window [lo, hi] keeps a candidate
// range (base, len) and halves it a fixed number of times (the table's
// widest window), branch-free: if g[base + len/2] <= E then base += len/2;
// len -= len/2.  Steps after len reaches 1 re-read g[base] and change
// nothing, so the result is the largest k in [lo, hi] with g[k] <= E (lo if
// none) -- the exact index.  The bracketing points' records (energy pair and
// FP32 cross sections) are read with 16-byte loads; the density is folded
// into the two weights, and the U species' terms are added before one
// compensated accumulation.  Slots past the material's end carry N = 0.
template <int W>
__device__ __forceinline__ void load_records(const float4* __restrict__ rec, int32_t p, float (&r0)[4 * W],
                                             float (&r1)[4 * W])
{
    const float4* q = rec + (int64_t)p * W;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const float4 a = __ldg(q + w), b = __ldg(q + W + w);
        r0[4 * w] = a.x; r0[4 * w + 1] = a.y; r0[4 * w + 2] = a.z; r0[4 * w + 3] = a.w;
        r1[4 * w] = b.x; r1[4 * w + 1] = b.y; r1[4 * w + 2] = b.z; r1[4 * w + 3] = b.w;
    }
}

template <typename V>
__device__ __forceinline__ V load_in(const V* p)
{
#if MCX_FAST_STREAM
    return __ldcs(p);
#else
    return __ldg(p);
#endif
}

__device__ __forceinline__ void store_out(double* p, double v)
{
#if MCX_FAST_STREAM
    __stcs(p, v);
#else
    *p = v;
#endif
}

template <int W, int U, int NC>
__device__ __forceinline__ void lookup_one(const Tables& t, int64_t j, const double* __restrict__ Ein,
                                           const int32_t* __restrict__ mat,
                                           const int32_t* __restrict__ perm, double* __restrict__ out)
{
    constexpr int NCMAX = NC;   // channels (a record holds up to 4 W - 2)
    static_assert(NC <= 4 * W - 2, "record too narrow for the channel count");
    const int nc = NC;
    const int64_t H1 = (int64_t)t.H + 1;
    const int64_t l = perm ? (int64_t)load_in(perm + j) : j;
    const double E = load_in(Ein + l);
    const int32_t m = load_in(mat + l);
    if (m < 0 || m >= t.n_materials || E != E) {
        for (int r = 0; r < nc; ++r) store_out(out + l * nc + r, __longlong_as_double(0x7ff8000000000000LL));
        return;
    }
    float hi[NCMAX], lo[NCMAX];
#pragma unroll
    for (int r = 0; r < NCMAX; ++r) hi[r] = lo[r] = 0.f;
    const float E_hi = (float)E;
    const float E_lo = (float)(E - (double)E_hi);
    const int64_t eb = search_key(E);
    const int32_t hb = t.H > 0 ? hash_bin(t, E, eb) : 0;
    const int32_t i0 = __ldg(t.moff + m), i1 = __ldg(t.moff + m + 1);
    for (int32_t i = i0; i < i1; i += U) {
        int32_t base[U], len[U];
        float N[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int32_t ii = i + u < i1 ? i + u : i1 - 1;
            const int4 e = __ldg(t.ment + ii);
            N[u] = i + u < i1 ? __int_as_float(e.w) : 0.f;
            if (t.H > 0) {
                const int32_t* h = t.hidx + (int64_t)e.z * H1 + hb;
                const int32_t wlo = __ldg(h);
                base[u] = e.x + wlo;
                len[u] = __ldg(h + 1) - wlo + 1;
            } else {
                base[u] = e.x;
                len[u] = e.y - 1;
            }
        }
        for (int st = 0; st < t.search_steps; ++st) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int32_t h = len[u] >> 1;
#if MCX_FAST_SKIP
                if (h > 0) {
                    if (ebits(__ldg(t.E + base[u] + h)) <= eb) base[u] += h;
                    len[u] -= h;
                }
#else
                if (ebits(__ldg(t.E + base[u] + h)) <= eb) base[u] += h;
                len[u] -= h;
#endif
            }
        }
        float part[NCMAX];
#pragma unroll
        for (int r = 0; r < NCMAX; ++r) part[r] = 0.f;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            float r0[4 * W], r1[4 * W];
            load_records<W>(t.frec, base[u], r0, r1);
            const float a = fmaxf((E_hi - r0[0]) + (E_lo - r0[1]), 0.f);
            const float b = fmaxf((r1[0] - E_hi) + (r1[1] - E_lo), 0.f);
#if MCX_FAST_FDIV
            const float nw = __fdividef(N[u], a + b);   // <= 2 ulp: within the budget above
#else
            const float nw = N[u] * __frcp_rn(a + b);
#endif
            const float w1 = nw * a, w0 = nw * b;
#pragma unroll
            for (int r = 0; r < NCMAX; ++r) {
#if MCX_FAST_FMA2
                part[r] = fmaf(w1, r1[2 + r], fmaf(w0, r0[2 + r], part[r]));
#else
                part[r] += fmaf(w0, r0[2 + r], w1 * r1[2 + r]);
#endif
            }
        }
#pragma unroll
        for (int r = 0; r < NCMAX; ++r) two_sum_acc(hi[r], lo[r], part[r]);
    }
#pragma unroll
    for (int r = 0; r < NCMAX; ++r) store_out(out + l * nc + r, (double)hi[r] + (double)lo[r]);
}

// Lookups are taken either with a grid-stride loop (work == nullptr) or, for
// binned orders, in chunks of kChunk consecutive positions that warps claim
// from the counter *work (zeroed before the launch): the whole GPU then
// sweeps the binned order from front to back, so the lookups in flight at
// any time sit in a narrow slice of (material, energy) and their tables stay
// in L2.  With a grid-stride loop, warps in small materials run ahead of
// those in large ones (up to 80x less work per lookup) and the lookups in
// flight spread over all materials and energies.
template <int W, int U, int NC>
__global__ void __launch_bounds__(256, MCX_FAST_MIN_BLOCKS) k_xs_lookup_fast(Tables t, int64_t n, const double* __restrict__ Ein,
                                                        const int32_t* __restrict__ mat,
                                                        const int32_t* __restrict__ perm,
                                                        double* __restrict__ out,
                                                        unsigned long long* __restrict__ work)
{
    if (work == nullptr) {
        for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
             j += (int64_t)gridDim.x * blockDim.x)
            lookup_one<W, U, NC>(t, j, Ein, mat, perm, out);
        return;
    }
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long base = 0ull;
        if (lane == 0) base = atomicAdd(work, (unsigned long long)kChunk);
        base = __shfl_sync(0xffffffffu, base, 0);
        if ((int64_t)base >= n) break;
#pragma unroll 1
        for (int r = 0; r < kChunk / 32; ++r) {
            const int64_t j = (int64_t)base + r * 32 + lane;
            if (j < n) lookup_one<W, U, NC>(t, j, Ein, mat, perm, out);
        }
    }
}

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int lookup_key(const SortParams& sp, double E, int32_t m)
{
    const float fb = (logf((float)E) - sp.ln_lo) * sp.scale;
    int b = fb >= 0.f ? (int)fb : 0;
    if (b >= sp.n_ebuckets) b = sp.n_ebuckets - 1;
    if (m < 0 || m >= sp.n_materials) m = 0;
    return m * sp.n_ebuckets + b;
}

__global__ void k_lookup_sort_count(SortParams sp, int64_t n, const double* __restrict__ E,
                                    const int32_t* __restrict__ mat, uint32_t* __restrict__ bins)
{
    extern __shared__ uint32_t hist[];
    const int nb = sp.n_materials * sp.n_ebuckets;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
         l += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&hist[lookup_key(sp, __ldg(E + l), __ldg(mat + l))], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
        if (hist[i]) atomicAdd(&bins[i], hist[i]);
}

// The same count with the histogram in global memory, for bin counts that do
// not fit in shared memory.
__global__ void k_lookup_sort_count_global(SortParams sp, int64_t n, const double* __restrict__ E,
                                           const int32_t* __restrict__ mat, uint32_t* __restrict__ bins)
{
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
         l += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&bins[lookup_key(sp, __ldg(E + l), __ldg(mat + l))], 1u);
}

__global__ void k_exclusive_scan(uint32_t* __restrict__ bins, int nb)
{
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t carry;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) carry = 0u;
    __syncthreads();
    for (int base = 0; base < nb; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < nb ? bins[i] : 0u;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            const int nw = blockDim.x >> 5;
            uint32_t s = threadIdx.x < nw ? warp_sums[threadIdx.x] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL, s, o);
                if (lane >= o) s += y;
            }
            if (threadIdx.x < nw) warp_sums[threadIdx.x] = s;
        }
        __syncthreads();
        const uint32_t before = (threadIdx.x >> 5) ? warp_sums[(threadIdx.x >> 5) - 1] : 0u;
        if (i < nb) bins[i] = carry + before + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += before + x;
        __syncthreads();
    }
}

__global__ void k_lookup_sort_scatter(SortParams sp, int64_t n, const double* __restrict__ E,
                                      const int32_t* __restrict__ mat, uint32_t* __restrict__ bins,
                                      int32_t* __restrict__ perm)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t l = base + threadIdx.x;
        const bool valid = l < n;
        const unsigned vm = __ballot_sync(FULL, valid);
        if (!valid) continue;
        const int key = lookup_key(sp, __ldg(E + l), __ldg(mat + l));
        const unsigned grp = __match_any_sync(vm, key);
        const int leader = __ffs(grp) - 1;
        uint32_t pos = 0u;
        if (lane == leader) pos = atomicAdd(&bins[key], (uint32_t)__popc(grp));
        pos = __shfl_sync(grp, pos, leader);
        perm[pos + __popc(grp & ((1u << lane) - 1u))] = (int32_t)l;
    }
}

}  // namespace

int launch_xs_lookup_fast(const Tables& t, int64_t n, const double* E, const int32_t* mat,
                          const int32_t* perm, double* out, int grid, cudaStream_t st,
                          unsigned long long* work)
{
    if (work && cudaMemsetAsync(work, 0, sizeof(unsigned long long), st) != cudaSuccess) return -1;
    // one instantiation per channel count: no work on unused record slots
    switch (t.n_ch) {
    case 1: k_xs_lookup_fast<1, kFastUnroll, 1><<<grid, 256, 0, st>>>(t, n, E, mat, perm, out, work); break;
    case 2: k_xs_lookup_fast<1, kFastUnroll, 2><<<grid, 256, 0, st>>>(t, n, E, mat, perm, out, work); break;
    case 3: k_xs_lookup_fast<2, kFastUnroll, 3><<<grid, 256, 0, st>>>(t, n, E, mat, perm, out, work); break;
    case 4: k_xs_lookup_fast<2, kFastUnroll, 4><<<grid, 256, 0, st>>>(t, n, E, mat, perm, out, work); break;
    case 5: k_xs_lookup_fast<2, kFastUnroll, 5><<<grid, 256, 0, st>>>(t, n, E, mat, perm, out, work); break;
    default: return -1;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_lookup_sort(const SortParams& sp, int64_t n, const double* E, const int32_t* mat,
                       uint32_t* bins, int32_t* perm, int grid, cudaStream_t st)
{
    const int nb = sp.n_materials * sp.n_ebuckets;
    if (cudaMemsetAsync(bins, 0, sizeof(uint32_t) * (size_t)(nb + 1), st) != cudaSuccess) return -1;
    if (nb <= kSmemBins)
        k_lookup_sort_count<<<grid, 512, sizeof(uint32_t) * nb, st>>>(sp, n, E, mat, bins);
    else
        k_lookup_sort_count_global<<<grid, 256, 0, st>>>(sp, n, E, mat, bins);
    k_exclusive_scan<<<1, 1024, 0, st>>>(bins, nb);
    k_lookup_sort_scatter<<<grid, 256, 0, st>>>(sp, n, E, mat, bins, perm);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace mcx
