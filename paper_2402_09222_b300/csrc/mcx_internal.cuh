// mcx_internal.cuh -- shared device-side definitions of libmcx (not part of
// the public ABI).  Everything here is written for sm_103a.
//
// Translation units that include the EXACT arithmetic helpers below
// (transport.cu, xs_exact.cu, adjoint.cu) are compiled with --fmad=false so
// that every FP64 expression is evaluated as written: one IEEE operation per
// operator, no fused multiply-add.  That is what makes grid indices, species
// choices and collision counts reproducible bit for bit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mcx.h"

namespace mcx {

// ---------------------------------------------------------------------------
// Bounds-checked builds (MCX_BOUNDS_CHECK=1, the library libmcx_bounds.so).
// Before the accesses that depend on caller data or on table contents -- a
// lookup index read from a processing order, a hash-grid search window, a
// particle slot read from an event queue, a queue append, a tally bin, a
// collision's species -- the kernels check the index.  A failed check is
// recorded in the translation unit's error word (site and index of the first
// failure; no __trap, no device assert) and the access is skipped or
// replaced by an in-range one, never made; the transport also stops its run
// with MCX_ERR_BOUNDS.  mcx_check_device and the transport run report it.
// Release builds compile every check away.
// ---------------------------------------------------------------------------
#ifndef MCX_BOUNDS_CHECK
#define MCX_BOUNDS_CHECK 0
#endif
enum BoundsSite : int {
    BC_PERM = 1,      // lookup index from a processing order outside [0, n)
    BC_WINDOW = 2,    // hash-grid search window outside the species' intervals
    BC_SLOT = 3,      // particle slot from an event queue outside [0, cap)
    BC_QUEUE = 4,     // event-queue append beyond its capacity
    BC_TALLY = 5,     // tally bin outside the tally arrays
    BC_SPECIES = 6,   // collision species outside the material
};
#if MCX_BOUNDS_CHECK
// first failed check of this translation unit: site << 56 | index (low 56 bits)
static __device__ unsigned long long g_bounds_err;
__device__ __forceinline__ bool bounds_check(bool ok, int site, long long idx)
{
    if (!ok)
        atomicCAS(&g_bounds_err, 0ull,
                  ((unsigned long long)site << 56) | ((unsigned long long)idx & ((1ull << 56) - 1ull)));
    return ok;
}
#define MCX_IN_BOUNDS(cond, site, idx) ::mcx::bounds_check((cond), (site), (long long)(idx))
// Host reader of the translation unit's error word (0: no failure); clears it.
#define MCX_BOUNDS_READER(fn)                                                           \
    unsigned long long fn()                                                             \
    {                                                                                   \
        unsigned long long v = 0ull, z = 0ull;                                          \
        if (cudaMemcpyFromSymbol(&v, g_bounds_err, sizeof(v)) != cudaSuccess) return 0ull; \
        if (v) cudaMemcpyToSymbol(g_bounds_err, &z, sizeof(z));                         \
        return v;                                                                       \
    }
#else
#define MCX_IN_BOUNDS(cond, site, idx) true
#define MCX_BOUNDS_READER(fn) \
    unsigned long long fn() { return 0ull; }
#endif

// ---------------------------------------------------------------------------
// Cross-section tables as seen by the kernels.
// Layout in HBM:
//   goff  int64 [S+1]     species s owns points [goff[s], goff[s+1])
//   E     f64   [P]       concatenated per-species energy grids
//   frec  f32x4 [P][w]    fast-path record of each point, 16-byte aligned:
//                         {g_hi, g_lo, s_0 .. s_{n_ch-1}, 0 ...} in w float4
//                         (w = 1 for n_ch <= 2, else 2), where (g_hi, g_lo) =
//                         (float(g), float(g - float(g))) is the energy as an
//                         unevaluated FP32 pair; the two bracketing points of a
//                         species are 2w consecutive float4
//   sigma f32|f64 [P][n_ch]  interleaved channels: the two points k, k+1 of
//                            one species are one contiguous 2*n_ch run
//   hidx  int32 [S][H+1]  hash grid: hidx[s][b] = grid index k of bin
//                         boundary b in species s (window of bin b is
//                         [hidx[s][b], hidx[s][b+1]])
//   hbound f64  [H+1]     bin boundaries, increasing, shared by all species
//   moff/msp/mden         CSR materials (offsets, species ids, densities)
// ---------------------------------------------------------------------------
struct Tables {
    int32_t n_species = 0;
    int32_t n_ch = 0;
    int32_t precision = MCX_FP64;
    int32_t n_materials = 0;
    int32_t max_mat_species = 0;
    int32_t ch_scatter = 0, ch_absorb = 1;
    int32_t ch_nu_fission = -1;   // -1: the tables carry no nu-fission channel
    int64_t n_points = 0;
    const int64_t* goff = nullptr;
    const double* E = nullptr;
    const double* winv = nullptr;   // per interval 1 / (g[k+1] - g[k])
    const double* slope = nullptr;  // per interval and channel (s[k+1] - s[k]) / (g[k+1] - g[k]) (transport)
    const double2* ttot = nullptr;  // per point {s_scatter + s_absorb, its interval slope} (transport)
    // Transport values as FP32 pairs (hi, lo = the rest), tpair_w float4 per
    // point: {g, total}, {total slope, absorption}, {absorption slope,
    // nu-fission}, {nu-fission slope, 0, 0}; and per material entry the
    // density as a pair.
    const float4* tpair = nullptr;
    int32_t tpair_w = 0;
    const float2* mden2 = nullptr;
    const float4* frec = nullptr;   // fast-path point records, frec_w float4 each
    int32_t frec_w = 0;
    const void* sigma = nullptr;
    const double* awr = nullptr;
    const double* inv_a1sq = nullptr;   // per species 1 / (A + 1)^2 (elastic kinematics)
    const int32_t* moff = nullptr;
    const int32_t* msp = nullptr;
    const double* mden = nullptr;
    const int4* ment = nullptr;   // per material entry: {first point, points, species, FP32 density bits}
    int32_t search_steps = 0;     // halvings that resolve the widest search window
    // hash grid (H == 0: none)
    int32_t H = 0;
    const int32_t* hidx = nullptr;
    const double* hbound = nullptr;
    float hash_ln_lo = 0.f;    // ln of hbound[0]
    float hash_scale = 0.f;    // H / (ln hbound[H] - ln hbound[0])
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the
// multiply-xor S-box with Weyl-sequence round keys.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += W0;
            k.y += W1;
        }
        const uint32_t lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
        const uint32_t lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Uniform number `n` of a history's stream.  Block n/2 of the stream keyed by
// (seed, problem) with counter (n/2, hist low word, hist high word, 0); even n
// uses words 0,1, odd n words 2,3.  Two words a, b map to (k + 1/2) 2^-52,
// k = (a >> 6) << 26 | (b >> 6): exact, strictly inside (0, 1).
__device__ __forceinline__ double uniform_at(uint2 key, uint64_t hist, uint32_t n)
{
    const uint4 w = philox4x32_10(
        make_uint4(n >> 1, (uint32_t)hist, (uint32_t)(hist >> 32), 0u), key);
    const uint32_t a = (n & 1u) ? w.z : w.x;
    const uint32_t b = (n & 1u) ? w.w : w.y;
    const uint64_t k = ((uint64_t)(a >> 6) << 26) | (uint64_t)(b >> 6);
    // (k + 0.5) 2^-52 = (2k + 1) 2^-53 exactly: built from the integer's bits
    // (leading one at bit p: exponent p - 53, the bits below it the
    // mantissa) instead of a conversion, an add and a multiply on B300's
    // 1/64-rate FP64 pipe.  Same value, bit for bit.
    const uint64_t m = (k << 1) | 1ull;
    const int p = 63 - __clzll((long long)m);
    const uint64_t mant = (m << (52 - p)) & 0x000FFFFFFFFFFFFFull;
    return __longlong_as_double((long long)(((uint64_t)(p - 53 + 1023) << 52) | mant));
}

__host__ __device__ __forceinline__ uint2 rng_key(uint64_t seed, uint32_t problem_id)
{
    return make_uint2((uint32_t)seed, (uint32_t)(seed >> 32) ^ problem_id);
}

// ---------------------------------------------------------------------------
// Grid search.  Energies are positive finite doubles, so their IEEE bit
// patterns, read as signed 64-bit integers, order exactly as the values do;
// comparing the integers runs on the integer pipes instead of B300's narrow
// FP64 pipe and gives the same decisions.  A negative or zero E orders below
// every grid point; NaN is mapped to k = 0 by the callers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t ebits(double x) { return __double_as_longlong(x); }

// Search key of a lookup energy: its bit pattern, or the lowest key for NaN
// (so a NaN energy takes grid index 0, as E < g[0] does).
__device__ __forceinline__ int64_t search_key(double E)
{
    return E != E ? (int64_t)0x8000000000000000LL : ebits(E);
}

// Largest k in [lo, hi] with g[k] <= E (lo if none).  Requires the answer of
// the full search to lie in [lo, hi].
__device__ __forceinline__ int64_t bsearch_window(const double* __restrict__ g, int64_t lo,
                                                  int64_t hi, int64_t eb)
{
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (ebits(__ldg(g + mid)) <= eb) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Hash bin of E: the b with hbound[b] <= E < hbound[b+1] (clamped to
// [0, H-1]).  The float logarithm only proposes a bin; two comparisons with
// the stored FP64 boundaries fix it, so the bin is exact whatever the
// rounding of logf.
__device__ __forceinline__ int32_t hash_bin(const Tables& t, double E, int64_t eb)
{
    const float lf = logf((float)E);
    float fb = (lf - t.hash_ln_lo) * t.hash_scale;
    int32_t b;
    if (!(fb >= 0.f)) b = 0;                       // also NaN, -inf, tiny E
    else if (fb >= (float)(t.H - 1)) b = t.H - 1;
    else b = (int32_t)fb;
    // at most a couple of steps: the float estimate is within a bin or two
    while (b > 0 && eb < ebits(__ldg(t.hbound + b))) --b;
    while (b < t.H - 1 && eb >= ebits(__ldg(t.hbound + b + 1))) ++b;
    return b;
}

// Grid index of species s for search key eb = search_key(E): the largest k
// in [0, n-2] with g[k] <= E, k = 0 below the grid or for NaN, n-2 at or
// above its top.
__device__ __forceinline__ int64_t species_index(const Tables& t, int32_t s, int64_t eb,
                                                 int32_t hbin)
{
    const int64_t base = __ldg(t.goff + s);
    const int64_t n = __ldg(t.goff + s + 1) - base;
    int64_t lo = 0, hi = n - 2;
    if (t.H > 0) {
        const int32_t* h = t.hidx + (int64_t)s * (t.H + 1) + hbin;
        lo = __ldg(h);
        hi = __ldg(h + 1);
        if (!MCX_IN_BOUNDS(lo >= 0 && lo <= hi && hi <= n - 2, BC_WINDOW, (int64_t)s * (t.H + 1) + hbin)) {
            lo = 0;
            hi = n - 2;
        }
    }
    return bsearch_window(t.E + base, lo, hi, eb);
}

// Exact FP32 -> FP64 widening with integer operations.  Table entries are
// validated finite and >= 0 at load time, so the sign bit is clear and the
// exponent field is below 255; a normal float 1.m * 2^(e-127) becomes the
// double with exponent field e + 896 and the 23 mantissa bits on top of the
// 52.  Zero and subnormals take the conversion instruction.  This keeps the
// widening off B300's FP64 pipe, which the FP64 arithmetic already saturates.
__device__ __forceinline__ double widen_f32(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = u >> 23;
    if (e == 0u) return u == 0u ? 0.0 : (double)f;
    const uint32_t hi = ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
    return __hiloint2double((int)hi, (int)(u << 29));
}

// Search window of species entry e = {first point, points, species, .} for
// hash bin hb, as a global first candidate and a candidate count.
__device__ __forceinline__ void search_window(const Tables& t, const int4& e, int32_t hb, int32_t& base,
                                              int32_t& len)
{
    if (t.H > 0) {
        const int32_t* h = t.hidx + (int64_t)e.z * ((int64_t)t.H + 1) + hb;
        const int32_t wlo = __ldg(h);
        base = e.x + wlo;
        len = __ldg(h + 1) - wlo + 1;
        if (!MCX_IN_BOUNDS(wlo >= 0 && len >= 1 && wlo + len <= e.y - 1, BC_WINDOW,
                           (int64_t)e.z * ((int64_t)t.H + 1) + hb)) {
            base = e.x;
            len = e.y - 1;
        }
    } else {
        base = e.x;
        len = e.y - 1;
    }
}

// One branch-free halving step of the fixed-step search: the candidate range
// (base, len) keeps the largest k with g[k] <= E; after t.search_steps steps
// len is 1 and base is that k (or the window start if none), exactly as
// bsearch_window finds it.
__device__ __forceinline__ void search_step(const double* __restrict__ E, int32_t& base, int32_t& len,
                                            int64_t eb)
{
    const int32_t h = len >> 1;
    if (ebits(__ldg(E + base + h)) <= eb) base += h;
    len -= h;
}

template <typename T>
__device__ __forceinline__ double sig_at(const void* sigma, int64_t i);

template <>
__device__ __forceinline__ double sig_at<double>(const void* sigma, int64_t i)
{
    return __ldg(static_cast<const double*>(sigma) + i);
}

template <>
__device__ __forceinline__ double sig_at<float>(const void* sigma, int64_t i)
{
    return widen_f32(__ldg(static_cast<const float*>(sigma) + i));
}

}  // namespace mcx
