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
// Records of 3-5 channels also carry r = float(1 / (g[k+1] - g[k])), and the
// weights are w1 = N sat(a r), w0 = N sat(b r) with a = E - g[k], b =
// g[k+1] - E from the pairs and sat() the saturation to [0, 1] (the clamp of
// energies outside the grid); records of 1-2 channels have no spare slot and
// divide instead: w1 = (N / (a + b)) a, w0 = (N / (a + b)) b.
// Error budget (u = 2^-24): the distances a, b carry ~2u; r half a unit, the
// two products one each, so a weight is within ~4u (~6u with the fast
// division: a + b one more, the division 2 ulp); the U species' 2U weighted
// terms of a group are added with fused multiply-adds (2U roundings, 8u at
// U = 4) and the groups are accumulated compensated (~1u).  All terms are
// non-negative, so the errors do not amplify: each output is within ~13u =
// 7.7e-7 (~15u = 9e-7 dividing) of the FP64 definition, under the 1e-6 bound
// (the largest measured on 1e8 outputs: 4.6e-7).
#include <cstdlib>

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
// Records of two float4 (3 to 5 channels) carry the FP32 reciprocal of their
// interval's width in their spare last slot, so the weights need no division.
#ifndef MCX_FAST_RINV
#define MCX_FAST_RINV 1
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
// Binned orders swept by chunk-claiming warps take the warp-cooperative form
// (k_xs_lookup_warp2); 0 keeps the per-lane form for them too.
#ifndef MCX_FAST_WARP
#define MCX_FAST_WARP 1
#endif
constexpr int kFastUnroll = MCX_FAST_UNROLL;
constexpr int kSmemBins = 12288;   // histograms up to this size count in shared memory
// Point records of 32 bytes loaded with one 256-bit load each.
#ifndef MCX_FAST_LD256
#define MCX_FAST_LD256 1
#endif
// Resident 256-thread blocks per SM of the two-lookups-per-lane form.
#ifndef MCX_FAST_PARK
#define MCX_FAST_PARK 1
#endif
#ifndef MCX_FAST2_MIN_BLOCKS
#define MCX_FAST2_MIN_BLOCKS 4
#endif
// The round-linear form has less work per species and more state per round:
// with 3 blocks per SM (80 registers, no spills) per 1e8 binned lookups
// 16.23 ms against 17.12 at 4 blocks (5 blocks: 18.11).
#ifndef MCX_LIN_MIN_BLOCKS
#define MCX_LIN_MIN_BLOCKS 3
#endif
static_assert(MCX_LIN_MIN_BLOCKS == kLinBlocksPerSm && MCX_FAST2_MIN_BLOCKS == kFastBlocksPerSm,
              "the launch grid sizes match the kernels' register caps");
// Each warp's 64 output rows of a round leave through shared memory: lane k
// of a store instruction writes value k of the round's rows laid end to end,
// so a row's values go out in one or two instructions whose lanes share its
// sectors, instead of one 8-byte store per value to 32 scattered rows (per
// 1e8 binned lookups the stores alone cost 7.3 ms that way).
#ifndef MCX_FAST_ROWSTAGE
#define MCX_FAST_ROWSTAGE 1
#endif
// Lookups a warp claims at a time in binned order: one 64-lookup round of the
// warp-cooperative form (24.9 ms per 1e8 against 25.2 for 128 and 25.5 for 256).
#ifndef MCX_FAST_CHUNK
#define MCX_FAST_CHUNK 64
#endif
constexpr int kChunk = MCX_FAST_CHUNK;
static_assert(kChunk % 64 == 0, "whole rounds of the warp-cooperative form");
// The round-linear form claims four rounds at a time: per 1e8 binned
// lookups 10.25 ms against 10.34 with two and 10.49 with one (its rounds are
// shorter, so the claim's round trip weighs more).
#ifndef MCX_LIN_CHUNK
#define MCX_LIN_CHUNK 256
#endif
static_assert(MCX_LIN_CHUNK % 64 == 0, "whole rounds of the warp-cooperative form");

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x)
{
    const float s = hi + x;
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += e;
}

// two_sum_acc on two independent sums at once with packed FP32 adds (each
// element rounds exactly as the scalar form does, so the results agree bit
// for bit).
#ifndef MCX_FAST_PACKED
#define MCX_FAST_PACKED 1
#endif
__device__ __forceinline__ void two_sum_acc2(float2& hi, float2& lo, float2 x)
{
#if MCX_FAST_PACKED
    // a - b as fma(b, -1, a): the product is exact, so one rounding, as in a - b
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 s = __fadd2_rn(hi, x);
    const float2 bp = __ffma2_rn(hi, m1, s);
    const float2 e = __fadd2_rn(__ffma2_rn(__ffma2_rn(bp, m1, s), m1, hi), __ffma2_rn(bp, m1, x));
    hi = s;
    lo = __fadd2_rn(lo, e);
#else
    two_sum_acc(hi.x, lo.x, x.x);
    two_sum_acc(hi.y, lo.y, x.y);
#endif
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

#if MCX_FAST_LD256
// 32-byte records (W = 2): each point is one 256-bit load (the table is
// allocated 256-byte aligned, so every record starts on a 32-byte boundary).
__device__ __forceinline__ void ld256(const float4* q, float (&r)[8])
{
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7])
        : "l"(q));
}

template <>
__device__ __forceinline__ void load_records<2>(const float4* __restrict__ rec, int32_t p, float (&r0)[8],
                                                float (&r1)[8])
{
    const float4* q = rec + (int64_t)p * 2;
    ld256(q, r0);
    ld256(q + 2, r1);
}
#endif

// Brings the 32-byte sector at p into L2 (no register result, no wait).
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

template <typename V>
__device__ __forceinline__ V load_in(const V* p)
{
#if MCX_FAST_STREAM
    return __ldcs(p);
#else
    return __ldg(p);
#endif
}

template <typename V>
__device__ __forceinline__ void store_stream(V* p, V v)
{
#if MCX_FAST_STREAM
    __stcs(p, v);
#else
    *p = v;
#endif
}

// An output channel from its compensated pair (hi, lo): the FP64 value
// hi + lo (exact), or that value rounded once to FP32.
__device__ __forceinline__ void store_out(double* p, float hi, float lo) { store_stream(p, (double)hi + (double)lo); }
__device__ __forceinline__ void store_out(float* p, float hi, float lo) { store_stream(p, hi + lo); }
template <typename OutT>
__device__ __forceinline__ OutT out_value(float hi, float lo);
template <>
__device__ __forceinline__ double out_value<double>(float hi, float lo) { return (double)hi + (double)lo; }
template <>
__device__ __forceinline__ float out_value<float>(float hi, float lo) { return hi + lo; }
__device__ __forceinline__ void store_nan(double* p) { store_stream(p, __longlong_as_double(0x7ff8000000000000LL)); }
__device__ __forceinline__ void store_nan(float* p) { store_stream(p, __int_as_float(0x7fc00000)); }

// One species' weighted terms added into part[]: the bracketing records r0
// (point k) and r1 (point k + 1), the lookup energy as the FP32 pair
// (E_hi, E_lo) and the FP32 density N.  Shared by every form of the fast
// lookup, so they agree bit for bit.
template <int W>
__device__ __forceinline__ void species_weights(const float (&r0)[4 * W], const float (&r1)[4 * W], float E_hi,
                                                float E_lo, float N, float& w0, float& w1)
{
    if constexpr (W == 2 && MCX_FAST_RINV) {
        // records of two float4 carry 1 / (g[k+1] - g[k]) in their last slot:
        // the fractions are the distances times it, saturated to [0, 1]
        // (which is the clamp of energies outside the grid), no division
        const float rw = r0[7];
        w1 = N * __saturatef(((E_hi - r0[0]) + (E_lo - r0[1])) * rw);
        w0 = N * __saturatef(((r1[0] - E_hi) + (r1[1] - E_lo)) * rw);
    } else {
        const float a = fmaxf((E_hi - r0[0]) + (E_lo - r0[1]), 0.f);
        const float b = fmaxf((r1[0] - E_hi) + (r1[1] - E_lo), 0.f);
#if MCX_FAST_FDIV
        const float nw = __fdividef(N, a + b);   // <= 2 ulp: within the budget above
#else
        const float nw = N * __frcp_rn(a + b);
#endif
        w1 = nw * a;
        w0 = nw * b;
    }
}

template <int W, int NC>
__device__ __forceinline__ void species_term(const float (&r0)[4 * W], const float (&r1)[4 * W], float E_hi,
                                             float E_lo, float N, float (&part)[NC])
{
    float w0, w1;
    species_weights<W>(r0, r1, E_hi, E_lo, N, w0, w1);
#pragma unroll
    for (int r = 0; r < NC; ++r) {
#if MCX_FAST_FMA2
        part[r] = fmaf(w1, r1[2 + r], fmaf(w0, r0[2 + r], part[r]));
#else
        part[r] += fmaf(w0, r0[2 + r], w1 * r1[2 + r]);
#endif
    }
}

// species_term for two lookups that share the species' records, their
// partial sums held as pairs (first lookup, second lookup): the channel
// updates as packed fused multiply-adds, each element the scalar form's.
#ifndef MCX_FAST_PACKED_TERM
#define MCX_FAST_PACKED_TERM 1
#endif
#ifndef MCX_FAST_PACKED_W
#define MCX_FAST_PACKED_W 1
#endif
template <int W, int NC>
__device__ __forceinline__ void species_term_pair(const float (&r0)[4 * W], const float (&r1)[4 * W], float Eh0,
                                                  float El0, float Eh1, float El1, float N, float2 (&part)[NC])
{
    static_assert(MCX_FAST_FMA2, "the pair form follows the two-FMA channel update");
#if MCX_FAST_PACKED_TERM && MCX_FAST_PACKED_W
    // species_weights for both lookups with packed operations: a - b as
    // fma(b, -1, a) (exact product, one rounding), the clamp per element
    float2 w0, w1;
    if constexpr (W == 2 && MCX_FAST_RINV) {
        const float2 m1 = make_float2(-1.f, -1.f);
        const float2 Eh = make_float2(Eh0, Eh1), El = make_float2(El0, El1);
        const float2 rw = make_float2(r0[7], r0[7]), Np = make_float2(N, N);
        float2 f1 = __fmul2_rn(__fadd2_rn(__ffma2_rn(make_float2(r0[0], r0[0]), m1, Eh),
                                          __ffma2_rn(make_float2(r0[1], r0[1]), m1, El)), rw);
        float2 f0 = __fmul2_rn(__fadd2_rn(__ffma2_rn(Eh, m1, make_float2(r1[0], r1[0])),
                                          __ffma2_rn(El, m1, make_float2(r1[1], r1[1]))), rw);
        f1 = make_float2(__saturatef(f1.x), __saturatef(f1.y));
        f0 = make_float2(__saturatef(f0.x), __saturatef(f0.y));
        w1 = __fmul2_rn(Np, f1);
        w0 = __fmul2_rn(Np, f0);
    } else {
        float w0a, w1a, w0b, w1b;
        species_weights<W>(r0, r1, Eh0, El0, N, w0a, w1a);
        species_weights<W>(r0, r1, Eh1, El1, N, w0b, w1b);
        w0 = make_float2(w0a, w0b);
        w1 = make_float2(w1a, w1b);
    }
#pragma unroll
    for (int r = 0; r < NC; ++r)
        part[r] = __ffma2_rn(w1, make_float2(r1[2 + r], r1[2 + r]),
                             __ffma2_rn(w0, make_float2(r0[2 + r], r0[2 + r]), part[r]));
#else
    float w0a, w1a, w0b, w1b;
    species_weights<W>(r0, r1, Eh0, El0, N, w0a, w1a);
    species_weights<W>(r0, r1, Eh1, El1, N, w0b, w1b);
#if MCX_FAST_PACKED_TERM
    const float2 w0 = make_float2(w0a, w0b), w1 = make_float2(w1a, w1b);
#pragma unroll
    for (int r = 0; r < NC; ++r)
        part[r] = __ffma2_rn(w1, make_float2(r1[2 + r], r1[2 + r]),
                             __ffma2_rn(w0, make_float2(r0[2 + r], r0[2 + r]), part[r]));
#else
#pragma unroll
    for (int r = 0; r < NC; ++r) {
        part[r].x = fmaf(w1a, r1[2 + r], fmaf(w0a, r0[2 + r], part[r].x));
        part[r].y = fmaf(w1b, r1[2 + r], fmaf(w0b, r0[2 + r], part[r].y));
    }
#endif
#endif
}

// species_term into one element of pair partial sums (lookups whose records differ).
template <int W, int NC, bool SECOND>
__device__ __forceinline__ void species_term_half(const float (&r0)[4 * W], const float (&r1)[4 * W], float E_hi,
                                                  float E_lo, float N, float2 (&part)[NC])
{
    float w0, w1;
    species_weights<W>(r0, r1, E_hi, E_lo, N, w0, w1);
#pragma unroll
    for (int r = 0; r < NC; ++r) {
        float& v = SECOND ? part[r].y : part[r].x;
        v = fmaf(w1, r1[2 + r], fmaf(w0, r0[2 + r], v));
    }
}

// ------------------------------------------------------------------------
// Round-linear sums (MCX_LOOKUP_LINEAR on a binned order).
//
// Inside one grid interval [g_k, g_k+1] a species' term
// N (s_k + (E - g_k) / (g_k+1 - g_k) (s_k+1 - s_k)) is linear in E, and the
// interpolant is continuous at every grid point.  A binned round's 64
// lookups lie in one material and a narrow range [E_min, E_max].  When that
// range holds no point of a species (strictly inside one interval) the
// species adds a + b x to the lookup at E, x = E - E_min, where a is its term
// at E_min and b its slope; when the range holds exactly one point g of the
// species it adds a + b x + db max(0, x - (g - E_min)), db the change of
// slope at g.  The a and b of such species are summed once per round (lanes
// over species) instead of once per lookup; each lookup then takes one
// multiply-add per channel, plus one per hinge (db) in its range.
//
// A species keeps the per-lookup form when the range holds two or more of
// its points, reaches outside its grid (the clamps are not linear), or when
// any channel's slope times the range width exceeds 1/kLinSlopeBound of its
// term at E_min: there a + b x could cancel.  Under that bound every term
// and partial sum stays within a small factor of the species' term, so the
// FP32 roundings cost a few ulps of the term, as in the per-lookup form;
// the totals are compensated sums as there.  The outputs differ from the
// per-lookup form's by rounding only, and they depend on which lookups share
// a round (the binned order within a bucket is not fixed).
constexpr float kLinSlopeBound = 16.f;
// species of a material whose grid index a warp keeps from one round of its
// chunk to the next (the round's E_min moves by about half a bucket, so the
// index stays or moves by one: two or three grid reads instead of a search)
constexpr int kLinKbCap = 384;
// rounds of materials with fewer species take the per-lookup form for all
// of them: the per-round reduction would cost more than it saves
#ifndef MCX_LIN_MIN_SPECIES
#define MCX_LIN_MIN_SPECIES 8
#endif

// 1 / (g_k+1 - g_k) in FP32 from the bracketing records: stored in the
// record's last slot by the two-float4 layout, computed from the energy
// pairs otherwise.
template <int W>
__device__ __forceinline__ float interval_rinv(const float (&r0)[4 * W], const float (&r1)[4 * W])
{
    if constexpr (W == 2 && MCX_FAST_RINV)
        return r0[7];
    else
        return __frcp_rn((r1[0] - r0[0]) + (r1[1] - r0[1]));
}

template <int W>
__device__ __forceinline__ void load_record(const float4* __restrict__ rec, int32_t p, float (&r)[4 * W])
{
#if MCX_FAST_LD256
    if constexpr (W == 2) {
        ld256(rec + (int64_t)p * 2, r);
        return;
    }
#endif
    const float4* q = rec + (int64_t)p * W;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const float4 a = __ldg(q + w);
        r[4 * w] = a.x; r[4 * w + 1] = a.y; r[4 * w + 2] = a.z; r[4 * w + 3] = a.w;
    }
}

// The linear pieces of one species for a round starting at E_ref (FP32 pair
// Erh + Erl) and spanning span16 / kLinSlopeBound: the term a at E_ref, the
// slope b of interval kb and, with d = 1, the change of slope db at point
// kb + 1 (whose energy pair comes back in g1h + g1l).  False when a slope
// breaks the cancellation bound.
template <int W, int NC>
__device__ __forceinline__ bool species_linear(const float4* __restrict__ rec, int32_t kb, int32_t d, float N,
                                               float Erh, float Erl, float span16, float (&a)[NC],
                                               float (&b)[NC], float (&db)[NC], float& g1h, float& g1l)
{
    float r0[4 * W], r1[4 * W];
    load_records<W>(rec, kb, r0, r1);
    g1h = r1[0];
    g1l = r1[1];
    float w0, w1;
    species_weights<W>(r0, r1, Erh, Erl, N, w0, w1);
    const float nr0 = N * interval_rinv<W>(r0, r1);
    bool ok = true;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        a[c] = fmaf(w1, r1[2 + c], w0 * r0[2 + c]);
        b[c] = nr0 * (r1[2 + c] - r0[2 + c]);
        ok = ok && fabsf(b[c]) * span16 <= a[c];
        db[c] = 0.f;
    }
    if (d == 1) {
        float r2[4 * W];
        load_record<W>(rec, kb + 2, r2);
        const float nr1 = N * interval_rinv<W>(r1, r2);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const float b1 = nr1 * (r2[2 + c] - r1[2 + c]);
            ok = ok && fabsf(b1) * span16 <= a[c];
            db[c] = b1 - b[c];
        }
    }
    return ok;
}

// One species of a lookup pair in the per-lookup form: records of interval b
// shared by both lookups, or (d > 0: the round's range holds d grid points)
// each lookup's own interval found among b .. b + d with its search key
// (read from *peb0, *peb1 only then); the terms go to pp.
template <int W, int NC>
__device__ __forceinline__ void species_pair(const Tables& t, int32_t b, int32_t d, float N,
                                             const volatile int64_t* peb0, const volatile int64_t* peb1, float Eh0,
                                             float El0, float Eh1, float El1, float2 (&pp)[NC])
{
    float r0[4 * W], r1[4 * W];
    if (d > 0) {
        const int64_t eb0 = *peb0, eb1 = *peb1;   // the lookups' search keys
        int32_t bb = b, len = d + 1;
        while (len > 1) search_step(t.E, bb, len, eb0);
        load_records<W>(t.frec, bb, r0, r1);
        species_term_half<W, NC, false>(r0, r1, Eh0, El0, N, pp);
        bb = b;
        len = d + 1;
        while (len > 1) search_step(t.E, bb, len, eb1);
        load_records<W>(t.frec, bb, r0, r1);
        species_term_half<W, NC, true>(r0, r1, Eh1, El1, N, pp);
    } else {
        load_records<W>(t.frec, b, r0, r1);
        species_term_pair<W, NC>(r0, r1, Eh0, El0, Eh1, El1, N, pp);
    }
}

template <int W, int U, int NC, typename OutT>
__device__ __forceinline__ void lookup_one(const Tables& t, int64_t n, int64_t j, const double* __restrict__ Ein,
                                           const int32_t* __restrict__ mat,
                                           const int32_t* __restrict__ perm, OutT* __restrict__ out,
                                           bool inb = false)
{
    constexpr int NCMAX = NC;   // channels (a record holds up to 4 W - 2)
    static_assert(NC <= 4 * W - 2, "record too narrow for the channel count");
    const int nc = NC;
    const int64_t l = perm ? (int64_t)load_in(perm + j) : j;
    if (perm && !MCX_IN_BOUNDS(l >= 0 && l < n, BC_PERM, l)) return;
    // inb: the inputs are given in the processing order
    const double E = load_in(Ein + (inb ? j : l));
    const int32_t m = load_in(mat + (inb ? j : l));
    if (m < 0 || m >= t.n_materials || E != E) {
        for (int r = 0; r < nc; ++r) store_nan(out + l * nc + r);
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
            search_window(t, e, hb, base[u], len[u]);
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
            species_term<W, NC>(r0, r1, E_hi, E_lo, N[u], part);
        }
#pragma unroll
        for (int r = 0; r < NCMAX; ++r) two_sum_acc(hi[r], lo[r], part[r]);
    }
#pragma unroll
    for (int r = 0; r < NCMAX; ++r) store_out(out + l * nc + r, hi[r], lo[r]);
}

// Lookups are taken either with a grid-stride loop (work == nullptr) or, for
// binned orders, in chunks of kChunk consecutive positions that warps claim
// from the counter *work (zeroed before the launch): the whole GPU then
// sweeps the binned order from front to back, so the lookups in flight at
// any time sit in a narrow slice of (material, energy) and their tables stay
// in L2.  With a grid-stride loop, warps in small materials run ahead of
// those in large ones (up to 80x less work per lookup) and the lookups in
// flight spread over all materials and energies.
template <int W, int U, int NC, typename OutT>
__global__ void __launch_bounds__(256, MCX_FAST_MIN_BLOCKS) k_xs_lookup_fast(Tables t, int64_t n, const double* __restrict__ Ein,
                                                        const int32_t* __restrict__ mat,
                                                        const int32_t* __restrict__ perm,
                                                        OutT* __restrict__ out,
                                                        unsigned long long* __restrict__ work)
{
    if (work == nullptr) {
        for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
             j += (int64_t)gridDim.x * blockDim.x)
            lookup_one<W, U, NC, OutT>(t, n, j, Ein, mat, perm, out);
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
            if (j < n) lookup_one<W, U, NC, OutT>(t, n, j, Ein, mat, perm, out);
        }
    }
}


// Warp-cooperative form for binned orders.  After binning, consecutive
// lookups share their material and lie in a narrow slice of energy, so for
// almost every species they fall in one grid interval.  A warp takes 64
// consecutive binned lookups per round (lane q: positions q and 32 + q) and
// works over groups of 32 species in two phases:
//  A. lanes over species: lane q finds, for species g0 + q, the grid index
//     k_lo of the round's lowest search key (hash window and fixed-step
//     search, exactly as lookup_one does per lookup) and, only where the
//     next grid point lies at or below the round's highest key (the slice
//     straddles grid points of that species; a few percent of species
//     visits), k_hi by a second search; otherwise k_hi = k_lo;
//  B. lanes over lookups: every lane walks the 32 species in groups of U,
//     takes k_lo, k_hi - k_lo and the density from lane q by shuffles, loads
//     the bracketing records once for both of its lookups and evaluates the
//     per-species term for each; where k_hi > k_lo each lookup searches its
//     own index inside [k_lo, k_hi] (the search is monotone in the key, so
//     the exact index lies there) and loads its own records.
// The window loads and searches are done once per warp and species instead
// of once per lookup, the record loads once per lane and species instead of
// once per lookup, and per lookup the species grouping and order of
// summation are lookup_one's: the outputs are bit-identical to it.  Rounds
// whose lookups mix materials or hold an invalid lookup (and the ragged
// tail) take lookup_one.  Measured per 1e8 binned lookups (355 x 11,303
// library, 68,400 hash bins): 25.6 ms against 28.4 ms for lookup_one in the
// same order; one lookup per lane 27.0 ms; 128-thread blocks (8 per SM) the
// same as 256; the records of 32 species staged
// in shared memory by cp.async 33.0 ms (the copies bypass L1, and the buffers
// shrink it); chunks of 256 or 512 lookups 27.9 and 29.3 ms; each lane's
// output rows and search keys parked in shared memory to relieve the
// registers 26.9 ms; FP32 -> FP64 widening of the outputs with integer
// operations instead of the FP64 pipe, no change; the rows and keys re-read
// from the permutation when needed instead of held, 62.8 ms.  With binning
// at about 192 lookups per bucket (22.8 ms), the lane's two lookups are
// paired in packed FP32 instructions (B300's two-wide add, multiply and
// fused multiply-add, each element rounded as the scalar operation): the
// compensated sums 22.6 ms, the channel updates 22.3 ms, the weights 22.2 ms;
// each lane's search keys and output rows parked in shared memory, so that
// the species loop spills half as much, 22.47 -> 22.27 ms on one box (with
// 3 blocks per SM and no spills at all, 23.58 ms against 22.24).  Later:
// each round's output rows leave through shared memory (MCX_FAST_ROWSTAGE,
// 21.8 -> 20.3 ms), and with the inputs in the binned order (inb) 18.4 ms.
// LIN: the round-linear sums above (the same prologue, searches and
// per-lookup body for the species they leave), 3 blocks per SM, warps
// claiming 256 lookups at a time: 10.25 ms per 1e8 on binned inputs.
template <int W, int U, int NC, typename OutT, bool LIN>
__global__ void __launch_bounds__(256, LIN ? MCX_LIN_MIN_BLOCKS : MCX_FAST2_MIN_BLOCKS) k_xs_lookup_warp2(Tables t, int64_t n, const double* __restrict__ Ein,
                                                         const int32_t* __restrict__ mat,
                                                         const int32_t* __restrict__ perm,
                                                         OutT* __restrict__ out,
                                                         unsigned long long* __restrict__ work, bool inb)
{
    static_assert(32 % U == 0, "species groups of U must tile the 32-species blocks");
    static_assert(!LIN || MCX_FAST_PARK, "the round-linear form keeps its per-lane sums in shared memory");
    const unsigned FULLM = 0xffffffffu;
    const int lane = threadIdx.x & 31;
#if MCX_FAST_PARK
    // each lane's search keys (read on the straddle path only) and output
    // rows (read at the end of the round) wait in shared memory, not in
    // registers through the species loop
    __shared__ int64_t s_park_eb[256 / 32][2][32];
    __shared__ int32_t s_park_l[256 / 32][2][32];
    volatile int64_t* park_eb0 = &s_park_eb[threadIdx.x >> 5][0][lane];
    volatile int64_t* park_eb1 = &s_park_eb[threadIdx.x >> 5][1][lane];
    volatile int32_t* park_l0 = &s_park_l[threadIdx.x >> 5][0][lane];
    volatile int32_t* park_l1 = &s_park_l[threadIdx.x >> 5][1][lane];
    // round-linear form: each lane's sums over its linear species, the terms
    // a as a compensated pair (slots c and NC + c), the slopes b (2 NC + c)
    __shared__ float s_lin[256 / 32][LIN ? 3 * NC : 1][32];
    volatile float* lin_acc = &s_lin[threadIdx.x >> 5][0][lane];
    // round-linear form: each species' grid index of the warp's previous
    // round (the next round of a chunk starts its search there)
    __shared__ int32_t s_kb[256 / 32][LIN ? kLinKbCap : 1];
#if MCX_FAST_ROWSTAGE
    __shared__ OutT s_rows[256 / 32][64 * NC];   // a round's output rows, end to end
#endif
#endif
    for (;;) {
        unsigned long long cbase = 0ull;
        constexpr int kCh = LIN ? MCX_LIN_CHUNK : kChunk;
        if (lane == 0) cbase = atomicAdd(work, (unsigned long long)kCh);
        cbase = __shfl_sync(FULLM, cbase, 0);
        if ((int64_t)cbase >= n) break;
        int32_t prev_mw = -1;   // material of the warp's previous round-linear round in this chunk
#pragma unroll 1
        for (int r = 0; r < kCh / 64; ++r) {
            const int32_t pm = prev_mw;
            prev_mw = -1;
            const int64_t j0 = (int64_t)cbase + r * 64 + lane, j1 = j0 + 32;
            bool in0 = j0 < n, in1 = j1 < n;
            int64_t l0 = 0, l1 = 0;
            double E0 = 0.0, E1 = 0.0;
            int32_t m0 = -1, m1 = -1;
            if (in0) {
                l0 = (int64_t)load_in(perm + j0);
                if (MCX_IN_BOUNDS(l0 >= 0 && l0 < n, BC_PERM, l0)) {
                    E0 = load_in(Ein + (inb ? j0 : l0));
                    m0 = load_in(mat + (inb ? j0 : l0));
                } else {
                    in0 = false;
                }
            }
            if (in1) {
                l1 = (int64_t)load_in(perm + j1);
                if (MCX_IN_BOUNDS(l1 >= 0 && l1 < n, BC_PERM, l1)) {
                    E1 = load_in(Ein + (inb ? j1 : l1));
                    m1 = load_in(mat + (inb ? j1 : l1));
                } else {
                    in1 = false;
                }
            }
            const int32_t mw = __shfl_sync(FULLM, m0, 0);
            const bool ok = in0 && in1 && m0 == mw && m1 == mw && mw >= 0 && mw < t.n_materials && E0 == E0 &&
                            E1 == E1;
            if (!__all_sync(FULLM, ok)) {
                if (in0) lookup_one<W, U, NC, OutT>(t, n, j0, Ein, mat, perm, out, inb);
                if (in1) lookup_one<W, U, NC, OutT>(t, n, j1, Ein, mat, perm, out, inb);
                continue;
            }
#if MCX_FAST_PARK
            int64_t eb_lo, eb_hi;
            {
                const int64_t e0 = search_key(E0), e1 = search_key(E1);
                *park_eb0 = e0;
                *park_eb1 = e1;
                *park_l0 = (int32_t)l0;
                *park_l1 = (int32_t)l1;
                eb_lo = e0 < e1 ? e0 : e1;
                eb_hi = e0 < e1 ? e1 : e0;
            }
#else
            const int64_t eb0 = search_key(E0), eb1 = search_key(E1);
            int64_t eb_lo = eb0 < eb1 ? eb0 : eb1, eb_hi = eb0 < eb1 ? eb1 : eb0;
#endif
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const int64_t a = __shfl_xor_sync(FULLM, eb_lo, o), b = __shfl_xor_sync(FULLM, eb_hi, o);
                eb_lo = a < eb_lo ? a : eb_lo;
                eb_hi = b > eb_hi ? b : eb_hi;
            }
            int32_t hb_lo = -1;   // hash bin of E_min, found when a search first needs it
            int32_t hb_hi = -1;
            float2 hi[NC], lo[NC];   // (lookup j0, lookup j1) per channel
#pragma unroll
            for (int c = 0; c < NC; ++c) hi[c] = lo[c] = make_float2(0.f, 0.f);
            const float Eh0 = (float)E0, El0 = (float)(E0 - (double)Eh0);
            const float Eh1 = (float)E1, El1 = (float)(E1 - (double)Eh1);
            const int32_t i0 = __ldg(t.moff + mw), i1 = __ldg(t.moff + mw + 1);
            // round-linear form: x = E - E_min per lookup, E_min as an FP32
            // pair, kLinSlopeBound times the round's energy range
            bool lin_round = false, any_lin = false;
            float2 x01 = make_float2(0.f, 0.f);
            float Erh = 0.f, Erl = 0.f, span16 = 0.f;
            if constexpr (LIN) {
                lin_round = i1 - i0 >= MCX_LIN_MIN_SPECIES;
                if (lin_round) {
                    const double Eref = __longlong_as_double(eb_lo);
                    Erh = (float)Eref;
                    Erl = (float)(Eref - (double)Erh);
                    // from the FP32 pairs: where a species is linear every energy of
                    // the round lies within two of its grid intervals of E_min, so
                    // the high parts' difference is exact (Sterbenz) and the sum
                    // rounds once, as the FP64 difference rounded to FP32 would
                    x01 = make_float2((Eh0 - Erh) + (El0 - Erl), (Eh1 - Erh) + (El1 - Erl));
                    span16 = kLinSlopeBound * (float)(__longlong_as_double(eb_hi) - Eref);
#pragma unroll
                    for (int q = 0; q < 3 * NC; ++q) lin_acc[32 * q] = 0.f;
                    prev_mw = mw;
                }
            }
            const bool reuse = LIN && lin_round && pm == mw;
            for (int32_t g0 = i0; g0 < i1; g0 += 32) {
                int32_t kb = 0, kd = 0;
                float Nq = 0.f;
                bool far = false;
                int4 e = make_int4(0, 0, 0, 0);
                if (g0 + lane < i1) {
                    e = __ldg(t.ment + g0 + lane);
                    Nq = __int_as_float(e.w);
                    const int32_t last = e.x + e.y - 2;
                    int32_t b0 = 0, ln0 = 1;
                    bool got = false;
                    int64_t gnx = 0;   // g[b0 + 1] as its bit pattern, where known
                    const int32_t si = g0 - i0 + lane;
                    if constexpr (LIN) {
                        // the largest k with g[k] <= E_min near the previous round's
                        // index kp: kp itself, kp + 1 or kp - 1, each decided exactly
                        if (reuse && si < kLinKbCap) {
                            const int32_t kp = s_kb[threadIdx.x >> 5][si];
                            if (kp >= e.x && kp <= last) {
                                const int64_t gk = ebits(__ldg(t.E + kp)), gk1 = ebits(__ldg(t.E + kp + 1));
                                if (gk <= eb_lo) {
                                    if (kp == last || eb_lo < gk1) {
                                        b0 = kp;
                                        gnx = gk1;
                                        got = true;
                                    } else if (kp + 1 == last) {
                                        b0 = last;   // g[last] <= E_min: the last interval
                                        got = true;
                                    } else {
                                        const int64_t gk2 = ebits(__ldg(t.E + kp + 2));
                                        if (eb_lo < gk2) {
                                            b0 = kp + 1;
                                            gnx = gk2;
                                            got = true;
                                        }
                                    }
                                } else if (kp > e.x) {
                                    if (ebits(__ldg(t.E + kp - 1)) <= eb_lo) {
                                        b0 = kp - 1;
                                        gnx = gk;
                                        got = true;
                                    }
                                }
                            }
                        }
                    }
                    if (!got) {
                        if (hb_lo < 0) hb_lo = t.H > 0 ? hash_bin(t, __longlong_as_double(eb_lo), eb_lo) : 0;
                        search_window(t, e, hb_lo, b0, ln0);
                        for (int st = 0; st < t.search_steps; ++st)
                            if (ln0 > 1) search_step(t.E, b0, ln0, eb_lo);
                        if (b0 < last) gnx = ebits(__ldg(t.E + b0 + 1));
                    }
                    kb = b0;
                    far = b0 < last && gnx <= eb_hi;
                    if constexpr (LIN)
                        if (lin_round && si < kLinKbCap) s_kb[threadIdx.x >> 5][si] = b0;
                }
                if (__any_sync(FULLM, far)) {
                    // kd: points of the species in (E_min, E_max].  With one (the
                    // common case) the largest k with g[k] <= E_max is kb + 1, known
                    // from g[kb + 2] > E_max (or kb + 1 the last interval); the
                    // search at E_max runs only for two or more
                    bool more = false;
                    if (far) {
                        if (kb + 1 == e.x + e.y - 2 || ebits(__ldg(t.E + kb + 2)) > eb_hi)
                            kd = 1;
                        else
                            more = true;
                    }
                    if (__any_sync(FULLM, more)) {
                        if (hb_hi < 0) hb_hi = t.H > 0 ? hash_bin(t, __longlong_as_double(eb_hi), eb_hi) : 0;
                        if (more) {
                            int32_t b1, ln1;
                            search_window(t, e, hb_hi, b1, ln1);
                            for (int st = 0; st < t.search_steps; ++st)
                                if (ln1 > 1) search_step(t.E, b1, ln1, eb_hi);
                            kd = b1 - kb;
                        }
                    }
                }
                bool linq = false;   // this lane's species is summed in linear form
                if constexpr (LIN) {
                    if (lin_round) {
                        float a[NC], b[NC], db[NC];
                        float xbp = 0.f;
                        bool hinge = false;
                        // one interval or one interior point in [E_min, E_max], inside the
                        // grid: the searches are exact (kb and kb + kd the largest k with
                        // g[k] <= E_min and <= E_max), so g[kb] <= E_min holds unless kb is
                        // the grid's first point, and E_max < g[kb + kd + 1] unless kb + kd
                        // is its last interval; only there are the points read
                        if (g0 + lane < i1 && kd <= 1 && (kb > e.x || ebits(__ldg(t.E + kb)) <= eb_lo) &&
                            (kb + kd < e.x + e.y - 2 || eb_hi <= ebits(__ldg(t.E + kb + kd + 1)))) {
                            float g1h, g1l;   // point kb + 1 as its FP32 pair
                            linq = species_linear<W, NC>(t.frec, kb, kd, Nq, Erh, Erl, span16, a, b, db, g1h, g1l);
                            if (linq) {
#pragma unroll
                                for (int c = 0; c < NC; ++c) {
                                    float h = lin_acc[32 * c], l = lin_acc[32 * (NC + c)];
                                    two_sum_acc(h, l, a[c]);
                                    lin_acc[32 * c] = h;
                                    lin_acc[32 * (NC + c)] = l;
                                    lin_acc[32 * (2 * NC + c)] = lin_acc[32 * (2 * NC + c)] + b[c];
                                }
                                hinge = kd == 1;
                                if (hinge) xbp = (g1h - Erh) + (g1l - Erl);   // as x01
                            }
                        }
                        any_lin = any_lin || __any_sync(FULLM, linq);
                        // each hinge's db max(0, x - x_g) for both lookups of every lane
                        unsigned hm = __ballot_sync(FULLM, hinge);
                        if (hm) {
                            float2 ph[NC];
#pragma unroll
                            for (int c = 0; c < NC; ++c) ph[c] = make_float2(0.f, 0.f);
                            while (hm) {
                                const int src = __ffs(hm) - 1;
                                hm &= hm - 1;
                                const float xb = __shfl_sync(FULLM, xbp, src);
                                const float2 h = make_float2(fmaxf(x01.x - xb, 0.f), fmaxf(x01.y - xb, 0.f));
#pragma unroll
                                for (int c = 0; c < NC; ++c) {
                                    const float dc = __shfl_sync(FULLM, db[c], src);
                                    ph[c] = __ffma2_rn(make_float2(dc, dc), h, ph[c]);
                                }
                            }
#pragma unroll
                            for (int c = 0; c < NC; ++c) two_sum_acc2(hi[c], lo[c], ph[c]);
                        }
                        // the other species per lookup, U at a time
                        unsigned fm = __ballot_sync(FULLM, g0 + lane < i1 && !linq);
                        int32_t prev = 0;
                        while (fm) {
                            float2 pp[NC];
#pragma unroll
                            for (int c = 0; c < NC; ++c) pp[c] = make_float2(0.f, 0.f);
#pragma unroll
                            for (int u = 0; u < U; ++u) {
                                const bool v = fm != 0u;
                                const int32_t src = v ? __ffs(fm) - 1 : prev;
                                prev = src;
                                fm &= fm - 1u;
                                const int32_t b = __shfl_sync(FULLM, kb, src);
                                const int32_t d = __shfl_sync(FULLM, kd, src);
                                const float Nu = __shfl_sync(FULLM, Nq, src);
                                species_pair<W, NC>(t, b, d, v ? Nu : 0.f, park_eb0, park_eb1, Eh0, El0, Eh1, El1,
                                                    pp);
                            }
#pragma unroll
                            for (int c = 0; c < NC; ++c) two_sum_acc2(hi[c], lo[c], pp[c]);
                        }
                        continue;
                    }
                }
                const int32_t gend = i1 < g0 + 32 ? i1 : g0 + 32;
                for (int32_t i = g0; i < gend; i += U) {
                    float2 pp[NC];   // partial sums (lookup j0, lookup j1)
#pragma unroll
                    for (int c = 0; c < NC; ++c) pp[c] = make_float2(0.f, 0.f);
                    const bool full = i + U <= i1;   // no padded slot in this group
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int32_t src = (full || i + u < i1 ? i + u : i1 - 1) - g0;
                        const int32_t b = __shfl_sync(FULLM, kb, src);
                        const int32_t d = __shfl_sync(FULLM, kd, src);
                        const float Nu = __shfl_sync(FULLM, Nq, src);
                        const float N = full || i + u < i1 ? Nu : 0.f;
                        float r0[4 * W], r1[4 * W];
                        if (d > 0) {
#if MCX_FAST_PARK
                            const int64_t eb0 = *park_eb0, eb1 = *park_eb1;
#endif
                            int32_t bb = b, len = d + 1;
                            while (len > 1) search_step(t.E, bb, len, eb0);
                            load_records<W>(t.frec, bb, r0, r1);
                            species_term_half<W, NC, false>(r0, r1, Eh0, El0, N, pp);
                            bb = b;
                            len = d + 1;
                            while (len > 1) search_step(t.E, bb, len, eb1);
                            load_records<W>(t.frec, bb, r0, r1);
                            species_term_half<W, NC, true>(r0, r1, Eh1, El1, N, pp);
                        } else {
                            load_records<W>(t.frec, b, r0, r1);
                            species_term_pair<W, NC>(r0, r1, Eh0, El0, Eh1, El1, N, pp);
                        }
                    }
#pragma unroll
                    for (int c = 0; c < NC; ++c) two_sum_acc2(hi[c], lo[c], pp[c]);
                }
            }
            if constexpr (LIN) {
                if (any_lin) {
                    // the round's sums over every lane's linear species (the
                    // butterfly leaves the same totals in every lane: each
                    // merge is commutative and the two-sum error is exact)
                    float Ah[NC], Al[NC], Bs[NC];
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        Ah[c] = lin_acc[32 * c];
                        Al[c] = lin_acc[32 * (NC + c)];
                        Bs[c] = lin_acc[32 * (2 * NC + c)];
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                        for (int c = 0; c < NC; ++c) {
                            const float h2 = __shfl_xor_sync(FULLM, Ah[c], o);
                            const float l2 = __shfl_xor_sync(FULLM, Al[c], o);
                            const float b2 = __shfl_xor_sync(FULLM, Bs[c], o);
                            const float s2 = Ah[c] + h2;
                            const float bp = s2 - Ah[c];
                            const float e2 = (Ah[c] - (s2 - bp)) + (h2 - bp);
                            Ah[c] = s2;
                            Al[c] = (Al[c] + l2) + e2;
                            Bs[c] = Bs[c] + b2;
                        }
                    }
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        two_sum_acc2(hi[c], lo[c], make_float2(Ah[c], Ah[c]));
                        lo[c] = __fadd2_rn(lo[c], make_float2(Al[c], Al[c]));
                        two_sum_acc2(hi[c], lo[c], __fmul2_rn(x01, make_float2(Bs[c], Bs[c])));
                    }
                }
            }
#if MCX_FAST_PARK && MCX_FAST_ROWSTAGE
            {
                OutT* rows = s_rows[threadIdx.x >> 5];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    rows[lane * NC + c] = out_value<OutT>(hi[c].x, lo[c].x);
                    rows[(32 + lane) * NC + c] = out_value<OutT>(hi[c].y, lo[c].y);
                }
                __syncwarp();
#pragma unroll
                for (int q = lane; q < 64 * NC; q += 32) {
                    const int row = q / NC;
                    const int64_t l = s_park_l[threadIdx.x >> 5][row >> 5][row & 31];
                    store_stream(out + l * NC + (q - row * NC), rows[q]);
                }
                __syncwarp();
            }
#else
#if MCX_FAST_PARK
            const int64_t r0 = *park_l0, r1 = *park_l1;
#else
            const int64_t r0 = l0, r1 = l1;
#endif
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                store_out(out + r0 * NC + c, hi[c].x, lo[c].x);
                store_out(out + r1 * NC + c, hi[c].y, lo[c].y);
            }
#endif
        }
    }
}

// Bin key of a lookup: material major, then the log-energy bucket.
// Two-level binning's stored keys: the bin key, and in bit 31 whether the
// lookup's material id is out of range; tfine keeps that bit in its bit 15.
constexpr uint32_t kKeyInvalid = 0x80000000u;
constexpr uint16_t kFineInvalid = 0x8000u;

__device__ __forceinline__ int lookup_key(const SortParams& sp, double E, int32_t m)
{
    const float fb = (logf((float)E) - sp.ln_lo) * sp.scale;
    int b = fb >= 0.f ? (int)fb : 0;
    if (b >= sp.n_ebuckets) b = sp.n_ebuckets - 1;
    if (m < 0 || m >= sp.n_materials) m = 0;
    return m * sp.n_ebuckets + b;
}

// ------------------------------------------------------------------------
// Staged binned lookup: a producer warp stages the records each chunk needs
// into shared memory with TMA bulk copies, eight consumer warps compute.
//
// The binned order puts 256 consecutive lookups in one material and a narrow
// slice of energy, so for each species of that material they need only the
// few grid points between the slice's lowest and highest energy.  Per chunk
// the producer reads the bin keys of the chunk's first and last lookup (the
// order is sorted by key, so they bound the chunk: one material, buckets
// b0..b1), widens the buckets' energy edges by a relative 1e-4 (the float
// logarithm of the bin key is within a few ulps), takes per species the
// union of the hash-grid windows over that energy range, and issues one
// cp.async.bulk for those point records into a shared-memory stage, arming
// the stage's mbarrier with the byte count.  A consumer whose own lookup is
// not in the chunk's material or energy range (or is invalid) takes the
// global-memory form for it.  One stage per block: while one block's producer
// stages, the SM's other blocks compute.
// Consumers wait on the mbarrier, search each species' few staged points and
// evaluate the same per-species terms as the global-memory form, in the same
// order, so the two agree bit for bit.  The search compares the energies'
// FP32 pairs (hi, lo) from the records: rounding to nearest is monotone, so
// hi (and on a tie of hi, lo) decides g <= E exactly whenever they differ;
// when both parts tie, the FP64 energy is read from global memory.  Two stages alternate: the producer fills one
// while the consumers work on the other.  A chunk that spans two materials,
// holds an invalid lookup or needs more points than a stage holds is done by
// the consumers with the global-memory form instead.
//
// Every wait is bounded in time; a wait that runs out sets *err, and the
// producer waits (again bounded) for its copies in flight before returning.
// ------------------------------------------------------------------------
constexpr int kStChunk = 256;                 // lookups per chunk (one per consumer thread)
constexpr int kStConsumerWarps = kStChunk / 32;
constexpr int kStThreads = 32 * (1 + kStConsumerWarps);
constexpr int kStMaxSpecies = 384;            // material entries a stage can describe
constexpr int kStMaxPoints = 1536;            // staged grid points (records) per stage
constexpr long long kStWaitCycles = 4000000000LL;   // ~2 s at 2 GHz
// Stages per block and blocks per SM (the blocks of an SM also overlap one
// another's staging and computing).  Measured per 1e8 binned lookups: 1
// stage x 3 blocks 33.7 ms, 2 x 2 34.2 ms, 1 x 2 43.9 ms, 3 x 1 53.0 ms --
// all slower than the global-memory form (28.4 ms), whose L1 already holds
// most records; the producer alone needs 12.2 ms, the consumers are the
// bound.  The staged form is kept as an option (MCX_LOOKUP_STAGED).
#ifndef MCX_STAGED_STAGES
#define MCX_STAGED_STAGES 1
#endif
#ifndef MCX_STAGED_BLOCKS
#define MCX_STAGED_BLOCKS 3
#endif
constexpr int kStStages = MCX_STAGED_STAGES;

enum { ST_NORMAL = 0, ST_FALLBACK = 1, ST_END = 2 };

struct StageInfo {
    long long base;   // first position of the chunk in the binned order
    int mode;
    int n_entries;    // species entries of the chunk's material
    int material;
    int pad;
    double E_min, E_max;   // every lookup staged for lies in [E_min, E_max]
};

template <int W>
struct StageLayout {
    static constexpr size_t kMeta = 0;                                     // int4 [kStMaxSpecies]
    static constexpr size_t kRec = kMeta + sizeof(int4) * kStMaxSpecies;   // float4 [kStMaxPoints * W]
    static constexpr size_t kInfo = kRec + sizeof(float4) * kStMaxPoints * W;   // StageInfo
    static constexpr size_t kBytes = (kInfo + sizeof(StageInfo) + 127) / 128 * 128;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}

// Wait for the phase of `parity` to complete, for at most `limit` cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit = kStWaitCycles)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// 1-D bulk copy global -> shared, completing on `bar` (both addresses 16-byte
// aligned, bytes a multiple of 16).
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ int warp_excl_scan(int v, int& total)
{
    const int lane = threadIdx.x & 31;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    total = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
}

// Producer: fill a stage with chunk `base` (the binned positions base ..
// base + kStChunk - 1).  Returns the bytes the stage's copies will deliver
// (0: nothing issued).
template <int W>
__device__ int producer_fill(const Tables& t, const SortParams& sp, int64_t n, const double* __restrict__ Ein,
                             const int32_t* __restrict__ mat, const int32_t* __restrict__ perm, long long base,
                             unsigned char* stage, uint64_t* full)
{
    using LY = StageLayout<W>;
    const int lane = threadIdx.x & 31;
    int4* meta = reinterpret_cast<int4*>(stage + LY::kMeta);
    float4* rec = reinterpret_cast<float4*>(stage + LY::kRec);
    StageInfo* info = reinterpret_cast<StageInfo*>(stage + LY::kInfo);
    // bin keys of the chunk's first and last lookup (lanes 0 and 1)
    int key = 0;
    if (lane < 2) {
        const int64_t j = lane == 0 ? (int64_t)base : ((int64_t)base + kStChunk - 1 < n ? (int64_t)base + kStChunk - 1 : n - 1);
        const int32_t l = __ldg(perm + j);
        key = MCX_IN_BOUNDS(l >= 0 && l < n, BC_PERM, l) ? lookup_key(sp, __ldg(Ein + l), __ldg(mat + l)) : -1;
    }
    const int k0 = __shfl_sync(0xffffffffu, key, 0), k1 = __shfl_sync(0xffffffffu, key, 1);
    const int m = k0 / sp.n_ebuckets, b0 = k0 % sp.n_ebuckets, b1 = k1 % sp.n_ebuckets;
    int mode = (k0 < 0 || k1 / sp.n_ebuckets != m || b1 < b0 || t.H == 0) ? ST_FALLBACK : ST_NORMAL;
    // the buckets' energy range, widened by a relative 1e-4
    const double E_min = b0 == 0 ? 0.0 : exp((double)sp.ln_lo + (double)b0 / (double)sp.scale) * (1.0 - 1e-4);
    const double E_max = b1 == sp.n_ebuckets - 1 ? __longlong_as_double(0x7ff0000000000000LL)
                                                 : exp((double)sp.ln_lo + (double)(b1 + 1) / (double)sp.scale) * (1.0 + 1e-4);
    int ne = 0, rec_total = 0;
    if (mode == ST_NORMAL) {
        const int32_t i0 = __ldg(t.moff + m);
        ne = __ldg(t.moff + m + 1) - i0;
        if (ne > kStMaxSpecies) mode = ST_FALLBACK;
        const int64_t H1 = (int64_t)t.H + 1;
        const int32_t hb_min = hash_bin(t, E_min, search_key(E_min));
        const int32_t hb_max = hash_bin(t, E_max, search_key(E_max));
        for (int q0 = 0; mode == ST_NORMAL && q0 < ne; q0 += 32) {
            const int q = q0 + lane;
            int L = 0, gp = 0, dens = 0;
            if (q < ne) {
                // every energy of bins hb_min..hb_max has its grid index in
                // [hidx[hb_min], hidx[hb_max + 1]]
                const int4 e = __ldg(t.ment + i0 + q);
                const int32_t* h = t.hidx + (int64_t)e.z * H1;
                const int32_t k_lo = __ldg(h + hb_min), k_hi = __ldg(h + hb_max + 1);
                gp = e.x + k_lo;
                L = k_hi - k_lo + 2;
                dens = e.w;
                if (!MCX_IN_BOUNDS(k_lo >= 0 && k_lo <= k_hi && k_hi <= e.y - 2, BC_WINDOW,
                                   (int64_t)e.z * H1 + hb_min))
                    L = kStMaxPoints + 1;   // no copy: the chunk takes the fallback below
            }
            int rsum;
            const int roff = warp_excl_scan(L, rsum);
            if (q < ne) meta[q] = make_int4(rec_total + roff, gp, L, dens);
            rec_total += rsum;
            if (rec_total > kStMaxPoints) mode = ST_FALLBACK;
        }
    }
    int bytes = 0;
    if (mode == ST_NORMAL) {
        bytes = rec_total * W * 16;
        if (lane == 0) mbar_expect_tx(full, (uint32_t)bytes);
        __syncwarp();
        for (int q = lane; q < ne; q += 32) {
            const int4 md = meta[q];
            tma_load_1d(rec + (size_t)md.x * W, t.frec + (int64_t)md.y * W, (uint32_t)(md.z * W * 16), full);
        }
        __syncwarp();
    }
    if (lane == 0) {
        info->base = base;
        info->mode = mode;
        info->n_entries = ne;
        info->material = m;
        info->E_min = E_min;
        info->E_max = E_max;
    }
    __syncwarp();
    return bytes;
}

// g <= E for the grid energy g of a staged record (FP32 pair rec.x, rec.y)
// and the lookup energy E (pair E_hi, E_lo, key eb); exact (see above).
__device__ __forceinline__ bool staged_le(float g_hi, float g_lo, float E_hi, float E_lo, int64_t eb,
                                          const double* __restrict__ g_exact)
{
    if (g_hi != E_hi) return g_hi < E_hi;
    if (g_lo != E_lo) return g_lo < E_lo;
    return ebits(__ldg(g_exact)) <= eb;
}

// Consumer: lookup `l` (energy E) of a staged chunk.
template <int W, int U, int NC, typename OutT>
__device__ __forceinline__ void consume_one(const Tables& t, const unsigned char* stage, int ne, int32_t l,
                                            double E, OutT* __restrict__ out)
{
    using LY = StageLayout<W>;
    const int4* meta = reinterpret_cast<const int4*>(stage + LY::kMeta);
    const float4* rec = reinterpret_cast<const float4*>(stage + LY::kRec);
    float hi[NC], lo[NC];
#pragma unroll
    for (int r = 0; r < NC; ++r) hi[r] = lo[r] = 0.f;
    const float E_hi = (float)E;
    const float E_lo = (float)(E - (double)E_hi);
    const int64_t eb = search_key(E);
    for (int i = 0; i < ne; i += U) {
        float part[NC];
#pragma unroll
        for (int r = 0; r < NC; ++r) part[r] = 0.f;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int ii = i + u < ne ? i + u : ne - 1;
            const int4 md = meta[ii];
            const float N = i + u < ne ? __int_as_float(md.w) : 0.f;
            // largest q in [0, L-2] with staged energy q <= E (0 if none)
            int q = 0;
            for (int qq = 1; qq <= md.z - 2; ++qq) {
                const float4 g = rec[(size_t)(md.x + qq) * W];
                if (staged_le(g.x, g.y, E_hi, E_lo, eb, t.E + md.y + qq)) q = qq;
                else break;
            }
            float r0[4 * W], r1[4 * W];
            const float4* p = rec + (size_t)(md.x + q) * W;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const float4 a = p[w], b = p[W + w];
                r0[4 * w] = a.x; r0[4 * w + 1] = a.y; r0[4 * w + 2] = a.z; r0[4 * w + 3] = a.w;
                r1[4 * w] = b.x; r1[4 * w + 1] = b.y; r1[4 * w + 2] = b.z; r1[4 * w + 3] = b.w;
            }
            species_term<W, NC>(r0, r1, E_hi, E_lo, N, part);
        }
#pragma unroll
        for (int r = 0; r < NC; ++r) two_sum_acc(hi[r], lo[r], part[r]);
    }
#pragma unroll
    for (int r = 0; r < NC; ++r) store_out(out + (int64_t)l * NC + r, hi[r], lo[r]);
}

template <int W, int U, int NC, typename OutT>
__global__ void __launch_bounds__(kStThreads, MCX_STAGED_BLOCKS) k_xs_lookup_staged(Tables t, SortParams sp, int64_t n,
                                                                    const double* __restrict__ Ein,
                                                                    const int32_t* __restrict__ mat,
                                                                    const int32_t* __restrict__ perm,
                                                                    OutT* __restrict__ out,
                                                                    unsigned long long* __restrict__ work,
                                                                    unsigned int* __restrict__ err,
                                                                    long long wait_cycles, int stall)
{
    using LY = StageLayout<W>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kStStages], empty[kStStages];
    // stages start on a 128-byte boundary (the launch adds 128 bytes of slack)
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kStConsumerWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == 0) {
        // ---- producer
        bool issued[kStStages];
        uint32_t issued_parity[kStStages];
        for (int s = 0; s < kStStages; ++s) {
            issued[s] = false;
            issued_parity[s] = 0u;
        }
        bool failed = false;
        for (int k = 0;; ++k) {
            const int s = k % kStStages, use = k / kStStages;
            if (use > 0) {
                if (!mbar_wait(&empty[s], (uint32_t)((use - 1) & 1), wait_cycles)) {
                    failed = true;
                    break;
                }
                issued[s] = false;   // the consumers waited for those copies before releasing
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            unsigned long long b = 0ull;
            if (lane == 0) b = atomicAdd(work, (unsigned long long)kStChunk);
            b = __shfl_sync(0xffffffffu, b, 0);
            unsigned char* stage = smem + (size_t)s * LY::kBytes;
            if ((int64_t)b >= n) {
                if (lane == 0) {
                    reinterpret_cast<StageInfo*>(stage + LY::kInfo)->mode = ST_END;
                    mbar_arrive(&full[s]);
                }
                break;
            }
            // test hook: the first chunk is claimed but never staged nor
            // signalled, so the consumers' wait on it runs out (no copies
            // are in flight for it)
            if (stall && k == 0) continue;
            const int bytes = producer_fill<W>(t, sp, n, Ein, mat, perm, (long long)b, stage, &full[s]);
            if (bytes > 0) {
                issued[s] = true;
                issued_parity[s] = (uint32_t)(use & 1);
            }
            if (lane == 0) mbar_arrive(&full[s]);
        }
        if (failed && lane == 0) atomicExch(err, 1u);
        // copies still in flight land before this block may exit (no later
        // phase of a slot with copies was started, so its parity is current)
        for (int s = 0; s < kStStages; ++s)
            if (issued[s] && !mbar_wait(&full[s], issued_parity[s]) && lane == 0) atomicExch(err, 1u);
        return;
    }
    // ---- consumers
    const int c = threadIdx.x - 32;
    for (int k = 0;; ++k) {
        const int s = k % kStStages, use = k / kStStages;
        if (!mbar_wait(&full[s], (uint32_t)(use & 1), wait_cycles)) {
            if (lane == 0) atomicExch(err, 1u);
            break;
        }
        const unsigned char* stage = smem + (size_t)s * LY::kBytes;
        const StageInfo info = *reinterpret_cast<const StageInfo*>(stage + LY::kInfo);
        if (info.mode == ST_END) break;
        const int64_t j = info.base + c;
        if (j < n) {
            const int32_t l = load_in(perm + j);
            if (MCX_IN_BOUNDS(l >= 0 && l < n, BC_PERM, l)) {
                const double E = load_in(Ein + l);
                const int32_t m = load_in(mat + l);
                // E >= E_min && E <= E_max is false for a NaN energy
                if (info.mode == ST_NORMAL && m == info.material && E >= info.E_min && E <= info.E_max)
                    consume_one<W, U, NC, OutT>(t, stage, info.n_entries, l, E, out);
                else
                    lookup_one<W, U, NC, OutT>(t, n, j, Ein, mat, perm, out);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

constexpr unsigned FULL = 0xffffffffu;

// Two-level binning: lookups per tile of passes 0 and A, lookups per
// sub-tile of pass B, fine bins per coarse bin (as bits), and the resident
// blocks per SM passes A and B are compiled for.  Per 1e8 lookups (binning
// time by CUDA events; 512-thread pass A unless noted): tile 8192 / sub-tile
// 8192 / 2 / 2 blocks 2.11 ms, 8192 / 4096 / 2 / 3 2.05 ms, 4096 / 8192 /
// 3 / 2 2.22 ms, 8192 / 8192 / 2 / 3 2.13 ms; at 128 lookups per bucket
// 8192 / 4096 / 2 / 3 2.08 ms and 16384 / 4096 / 1 / 3 with a 1024-thread
// pass A 2.02 ms (the setting: half the per-tile work per lookup, and a
// tile scan that covers 4096 coarse bins, every bin count's); the one-level
// sort 2.63 ms on a like box.
#ifndef MCX_BIN2_TILE
#define MCX_BIN2_TILE 16384
#endif
#ifndef MCX_BIN2_SUB
#define MCX_BIN2_SUB 4096
#endif
#ifndef MCX_BIN2_A_BLOCKS
#define MCX_BIN2_A_BLOCKS 1
#endif
#ifndef MCX_BIN2_B_BLOCKS
#define MCX_BIN2_B_BLOCKS 3
#endif
constexpr int kBinTile = MCX_BIN2_TILE;
constexpr int kBinSub = MCX_BIN2_SUB;
constexpr int kBinFineBits = 9;


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
// Bin key of lookup l for a warp-wide binning step (keys of lanes past n are
// negative and distinct), and whether two neighbouring lanes share a key: only
// then do the kernels below aggregate equal keys with a warp match, which
// costs more than the atomics it saves on well-spread keys.
__device__ __forceinline__ int warp_bin_key(const SortParams& sp, const double* E, const int32_t* mat,
                                            int64_t l, int64_t n, int lane, bool& dup)
{
    const int key = l < n ? lookup_key(sp, __ldg(E + l), __ldg(mat + l)) : -1 - lane;
    const int prev = __shfl_up_sync(FULL, key, 1);
    dup = __any_sync(FULL, lane > 0 && prev == key);
    return key;
}

__global__ void k_lookup_sort_count_global(SortParams sp, int64_t n, const double* __restrict__ E,
                                           const int32_t* __restrict__ mat, uint32_t* __restrict__ bins)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t l = base + threadIdx.x;
        const unsigned vm = __ballot_sync(FULL, l < n);
        bool dup;
        const int key = warp_bin_key(sp, E, mat, l, n, lane, dup);
        if (l >= n) continue;
        if (!dup) {
            atomicAdd(&bins[key], 1u);
        } else {
            const unsigned grp = __match_any_sync(vm, key);
            if (lane == __ffs(grp) - 1) atomicAdd(&bins[key], (uint32_t)__popc(grp));
        }
    }
}

// Exclusive scan of the bin counters in two launches over parts of `seg`
// consecutive bins: each part sums its bins into part[], then each part adds
// the sums of the parts before it and scans its own bins from there.

// Sum of v over a block of 1024 threads (valid in thread 0).
__device__ __forceinline__ uint32_t block_sum_1024(uint32_t v, uint32_t* red)
{
    v = __reduce_add_sync(FULL, v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    uint32_t s = 0u;
    if (threadIdx.x < 32) s = __reduce_add_sync(FULL, red[threadIdx.x]);
    return s;
}

__global__ void __launch_bounds__(1024) k_scan_part_sums(const uint32_t* __restrict__ bins, int nb, int seg,
                                                         uint32_t* __restrict__ part)
{
    __shared__ uint32_t red[32];
    const int i0 = blockIdx.x * seg;
    const int i1 = min(nb, i0 + seg);
    uint32_t v = 0u;
    for (int i = i0 + threadIdx.x; i < i1; i += 1024) v += bins[i];
    v = block_sum_1024(v, red);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}

__global__ void __launch_bounds__(1024) k_scan_parts(uint32_t* __restrict__ bins, int nb, int seg,
                                                     const uint32_t* __restrict__ part)
{
    __shared__ uint32_t red[32];
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // offset of this part: the sum of the parts before it
    uint32_t v = 0u;
    for (int j = threadIdx.x; j < (int)blockIdx.x; j += 1024) v += part[j];
    v = block_sum_1024(v, red);
    if (threadIdx.x == 0) carry = v;
    __syncthreads();
    const int i0 = blockIdx.x * seg;
    const int i1 = min(nb, i0 + seg);
    for (int base = i0; base < i1; base += 1024) {
        const int i = base + threadIdx.x;
        const uint32_t c = i < i1 ? bins[i] : 0u;
        uint32_t x = c;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t s = warp_sums[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL, s, o);
                if (lane >= o) s += y;
            }
            warp_sums[lane] = s;
        }
        __syncthreads();
        const uint32_t before = warp ? warp_sums[warp - 1] : 0u;
        if (i < i1) bins[i] = carry + before + x - c;
        __syncthreads();
        if (threadIdx.x == 1023) carry += before + x;
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
        bool dup;
        const int key = warp_bin_key(sp, E, mat, l, n, lane, dup);
        if (!valid) continue;
        if (!dup) {
            perm[atomicAdd(&bins[key], 1u)] = (int32_t)l;
            continue;
        }
        const unsigned grp = __match_any_sync(vm, key);
        const int leader = __ffs(grp) - 1;
        uint32_t pos = 0u;
        if (lane == leader) pos = atomicAdd(&bins[key], (uint32_t)__popc(grp));
        pos = __shfl_sync(grp, pos, leader);
        perm[pos + __popc(grp & ((1u << lane) - 1u))] = (int32_t)l;
    }
}

// ------------------------------------------------------ two-level binning
// The same binning for large batches without a global atomic per lookup.
// The bin key splits into a coarse bin (key >> kBinFineBits, at most a few
// thousand) and a fine bin (the low bits).  Pass 0 counts each tile's
// lookups per coarse bin in shared memory into cnt[coarse * n_tiles + tile];
// an exclusive scan of that matrix gives every (coarse bin, tile) its place.
// Pass A re-reads each tile, takes places within the tile's runs by
// shared-memory atomics and writes the lookup index and its fine bin there
// (a tile's runs are short and filled at once, so L2 merges the partial
// writes).  Pass B gives each coarse bin to one block, which counts its fine
// bins in shared memory and scatters the indices into the final order.
__global__ void __launch_bounds__(512) k_bin2_count(SortParams sp, int64_t n, const double* __restrict__ E,
                                                   const int32_t* __restrict__ mat, int n_coarse, int n_tiles,
                                                   uint32_t* __restrict__ cnt, uint32_t* __restrict__ keys)
{
    extern __shared__ uint32_t h[];   // [n_coarse]
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        for (int i = threadIdx.x; i < n_coarse; i += blockDim.x) h[i] = 0u;
        __syncthreads();
        const int64_t base = (int64_t)tile * kBinTile;
        for (int k = threadIdx.x; k < kBinTile; k += blockDim.x) {
            const int64_t l = base + k;
            if (l < n) {
                const int32_t m = __ldg(mat + l);
                const uint32_t key = (uint32_t)lookup_key(sp, __ldg(E + l), m);
                // bit 31: a material id outside [0, n_materials) (binned with material 0)
                keys[l] = key | (m < 0 || m >= sp.n_materials ? kKeyInvalid : 0u);
                atomicAdd(&h[key >> kBinFineBits], 1u);
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n_coarse; i += blockDim.x) cnt[(int64_t)i * n_tiles + tile] = h[i];
        __syncthreads();
    }
}

// Exclusive scan, in place, of a[0, m) in shared memory for m <= 4 x
// blockDim.x (blockDim.x a multiple of 32, at most 1024); every thread calls it.
__device__ __forceinline__ void smem_exclusive_scan(uint32_t* a, int m, uint32_t* warp_sums)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int i0 = threadIdx.x * 4;
    uint32_t v[4], t = 0u;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v[q] = i0 + q < m ? a[i0 + q] : 0u;
        t += v[q];
    }
    uint32_t x = t;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? warp_sums[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) warp_sums[lane] = w;
    }
    __syncthreads();
    uint32_t run = (warp ? warp_sums[warp - 1] : 0u) + x - t;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (i0 + q < m) a[i0 + q] = run;
        run += v[q];
    }
    __syncthreads();
}

#ifndef MCX_BIN2_A_THREADS
#define MCX_BIN2_A_THREADS 1024
#endif
constexpr int kBin2Threads = MCX_BIN2_A_THREADS;
constexpr int kBin2PerThread = kBinTile / kBin2Threads;

// Pass A, one tile at a time: the tile's lookups are ranked by coarse bin in
// shared memory, staged in that order, and written out as contiguous runs.
// The fine bin goes out with the invalid-material bit of the key (bit 15).
// CARRY: each lookup's energy travels with its index into the coarse order
// (tE), so that the final order can hand it to the lookup in sequence
// instead of through the permutation; the energies are loaded in index
// order and staged in slot order in place of the keys, which the write-out
// re-reads from the tile's (cache-hot) window.  The material is not carried:
// pass B derives it from the bin.
template <bool CARRY>
__global__ void __launch_bounds__(kBin2Threads, MCX_BIN2_A_BLOCKS) k_bin2_scatter(int64_t n, const uint32_t* __restrict__ keys,
                                                              int n_coarse, int n_tiles,
                                                              const uint32_t* __restrict__ place,
                                                              int32_t* __restrict__ tidx,
                                                              uint16_t* __restrict__ tfine,
                                                              const double* __restrict__ E,
                                                              double* __restrict__ tE)
{
    extern __shared__ uint32_t sm[];
    uint32_t* cur = sm;                                    // [n_coarse] first place of (bin, tile)
    uint32_t* lst = sm + n_coarse;                         // [n_coarse] tile-local counts, then starts
    int32_t* sidx = reinterpret_cast<int32_t*>(sm + 2 * n_coarse);   // [kBinTile] staged indices
    // [kBinTile] staged keys, or with CARRY staged energies (8-byte aligned:
    // 2 n_coarse + kBinTile words precede them, an even count)
    uint32_t* skey = reinterpret_cast<uint32_t*>(sidx + kBinTile);
    double* sE = reinterpret_cast<double*>(sidx + kBinTile);
    __shared__ uint32_t warp_sums[32];
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        for (int i = threadIdx.x; i < n_coarse; i += blockDim.x) {
            cur[i] = place[(int64_t)i * n_tiles + tile];
            lst[i] = 0u;
        }
        __syncthreads();
        const int64_t base = (int64_t)tile * kBinTile;
        const int cnt = n - base < kBinTile ? (int)(n - base) : kBinTile;
        uint32_t key[kBin2PerThread], rk[kBin2PerThread];
#pragma unroll
        for (int j = 0; j < kBin2PerThread; ++j) {
            const int k = threadIdx.x + j * kBin2Threads;
            key[j] = 0u;
            rk[j] = 0u;
            if (k < cnt) {
                key[j] = __ldg(keys + base + k);
                rk[j] = atomicAdd(&lst[(key[j] & ~kKeyInvalid) >> kBinFineBits], 1u);
            }
        }
        __syncthreads();
        smem_exclusive_scan(lst, n_coarse, warp_sums);
#pragma unroll
        for (int j = 0; j < kBin2PerThread; ++j) {
            const int k = threadIdx.x + j * kBin2Threads;
            if (k < cnt) {
                const uint32_t slot = lst[(key[j] & ~kKeyInvalid) >> kBinFineBits] + rk[j];
                sidx[slot] = (int32_t)(base + k);
                if constexpr (CARRY)
                    sE[slot] = load_in(E + base + k);
                else
                    skey[slot] = key[j];
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kBin2PerThread; ++j) {
            const int k = threadIdx.x + j * kBin2Threads;
            if (k < cnt) {
                const int32_t ix = sidx[k];
                const uint32_t kk = CARRY ? __ldg(keys + ix) : skey[k];
                const uint32_t c = (kk & ~kKeyInvalid) >> kBinFineBits;
                const uint32_t pos = cur[c] + ((uint32_t)k - lst[c]);
                tidx[pos] = ix;
                tfine[pos] = (uint16_t)((kk & ((1u << kBinFineBits) - 1u)) | (kk & kKeyInvalid ? kFineInvalid : 0u));
                if constexpr (CARRY) tE[pos] = sE[k];
            }
        }
        __syncthreads();
    }
}

// Pass B: coarse bin c holds places [place[c * n_tiles], place[(c + 1) *
// n_tiles]) (n for the last), the same range in the final order.  One block
// per coarse bin counts its fine bins, then takes the range in sub-tiles of
// kBinSub: each is ranked by fine bin in shared memory, staged, and written
// out as contiguous runs.  CARRY: the energies in the coarse order (tE) are
// staged with their indices and follow them into the final order (Eb); the
// material comes from the bin, (c * 512 + fine bin) / n_ebuckets, or -1 for
// a lookup whose material id was out of range (Mb).
constexpr int kBin2FineThreads = 1 << kBinFineBits;    // one fine bin per thread
// With the carry, pass B takes larger sub-tiles so that each fine bin's run
// per sub-tile is longer (fewer partially written sectors at the run ends):
// blocks of MCX_BIN2_B_CARRY_THREADS threads (the first 512 also keep one
// fine bin each), MCX_BIN2_B_CARRY_SUB lookups per sub-tile.
#ifndef MCX_BIN2_B_CARRY_THREADS
#define MCX_BIN2_B_CARRY_THREADS 1024
#endif
#ifndef MCX_BIN2_B_CARRY_SUB
#define MCX_BIN2_B_CARRY_SUB 8192
#endif
#ifndef MCX_BIN2_B_CARRY_BLOCKS
#define MCX_BIN2_B_CARRY_BLOCKS 1
#endif
template <bool CARRY>
struct Bin2Fine {
    static constexpr int kThreads = CARRY ? MCX_BIN2_B_CARRY_THREADS : kBin2FineThreads;
    static constexpr int kSub = CARRY ? MCX_BIN2_B_CARRY_SUB : kBinSub;
    static constexpr int kBlocks = CARRY ? MCX_BIN2_B_CARRY_BLOCKS : MCX_BIN2_B_BLOCKS;
    static constexpr int kPer = kSub / kThreads;
    static_assert(kSub % kThreads == 0 && kThreads >= kBin2FineThreads && kThreads <= 1024, "pass B shape");
    static_assert(kSub <= (1 << (32 - kBinFineBits)), "rank and fine bin share a word");
};
template <bool CARRY>
__global__ void __launch_bounds__(Bin2Fine<CARRY>::kThreads, Bin2Fine<CARRY>::kBlocks) k_bin2_fine(int64_t n, int n_coarse, int n_tiles,
                                                               const uint32_t* __restrict__ place,
                                                               const int32_t* __restrict__ tidx,
                                                               const uint16_t* __restrict__ tfine,
                                                               int32_t* __restrict__ perm,
                                                               const double* __restrict__ tE, int n_ebuckets,
                                                               double* __restrict__ Eb, int32_t* __restrict__ Mb)
{
    constexpr int F = kBin2FineThreads;
    constexpr int T = Bin2Fine<CARRY>::kThreads, kSub = Bin2Fine<CARRY>::kSub, kPer = Bin2Fine<CARRY>::kPer;
    constexpr uint16_t kFineMask = (1u << kBinFineBits) - 1u;
    const bool bin_owner = threadIdx.x < F;            // thread keeps fine bin threadIdx.x
    extern __shared__ uint32_t sm[];
    uint32_t* fcur = sm;                               // [F] next place of each fine bin in the range
    uint32_t* lst = sm + F;                            // [F] sub-tile counts, then starts
    int32_t* sidx = reinterpret_cast<int32_t*>(sm + 2 * F);            // [kSub] staged indices
    // CARRY: [kSub] staged energies (2 F + kSub words precede them: even)
    double* sE = reinterpret_cast<double*>(sidx + kSub);
    uint16_t* sfine = reinterpret_cast<uint16_t*>(sE + (CARRY ? kSub : 0));   // [kSub] staged fine bins
    __shared__ uint32_t warp_sums[32];
    for (int c = blockIdx.x; c < n_coarse; c += gridDim.x) {
        const int64_t s0 = place[(int64_t)c * n_tiles];
        const int64_t s1 = c + 1 < n_coarse ? (int64_t)place[(int64_t)(c + 1) * n_tiles] : n;
        if (bin_owner) fcur[threadIdx.x] = 0u;
        __syncthreads();
        for (int64_t e = s0 + threadIdx.x; e < s1; e += T) atomicAdd(&fcur[__ldg(tfine + e) & kFineMask], 1u);
        __syncthreads();
        smem_exclusive_scan(fcur, F, warp_sums);
        for (int64_t sub = s0; sub < s1; sub += kSub) {
            const int cnt = s1 - sub < kSub ? (int)(s1 - sub) : kSub;
            if (bin_owner) lst[threadIdx.x] = 0u;
            __syncthreads();
            // per element its rank within its fine bin (< kSub) above the
            // fine bin's kBinFineBits bits
            uint32_t fr[kPer];
            int32_t ix[kPer];
            uint16_t tf[kPer];
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
                const int k = threadIdx.x + j * T;
                fr[j] = 0u;
                ix[j] = 0;
                tf[j] = 0;
                if (k < cnt) {
                    tf[j] = __ldg(tfine + sub + k);
                    const uint32_t fb = tf[j] & kFineMask;
                    ix[j] = __ldg(tidx + sub + k);
                    fr[j] = (atomicAdd(&lst[fb], 1u) << kBinFineBits) | fb;
                }
            }
            __syncthreads();
            // this sub-tile's count of fine bin threadIdx.x
            const uint32_t mine = bin_owner ? lst[threadIdx.x] : 0u;
            __syncthreads();
            smem_exclusive_scan(lst, F, warp_sums);
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
                const int k = threadIdx.x + j * T;
                if (k < cnt) {
                    const uint32_t fb = fr[j] & ((1u << kBinFineBits) - 1u);
                    const uint32_t slot = lst[fb] + (fr[j] >> kBinFineBits);
                    sidx[slot] = ix[j];
                    sfine[slot] = tf[j];
                    if constexpr (CARRY) sE[slot] = load_in(tE + sub + k);
                }
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
                const int k = threadIdx.x + j * T;
                if (k < cnt) {
                    const uint32_t tfk = sfine[k];
                    const uint32_t fb = tfk & kFineMask;
                    const int64_t pos = s0 + fcur[fb] + ((uint32_t)k - lst[fb]);
                    perm[pos] = sidx[k];
                    if constexpr (CARRY) {
                        Eb[pos] = sE[k];
                        Mb[pos] = (tfk & kFineInvalid) ? -1
                                                       : (int32_t)((((uint32_t)c << kBinFineBits) | fb) /
                                                                   (uint32_t)n_ebuckets);
                    }
                }
            }
            __syncthreads();
            if (bin_owner) fcur[threadIdx.x] += mine;
            __syncthreads();
        }
    }
}

// CARRY on the one-level path: the energies and materials in the binned
// order by a gather through the permutation (batches below the two-level
// size, whose inputs mostly sit in L2); a material id outside [0,
// n_materials) becomes -1, as the two-level path writes it.
__global__ void k_gather_inputs(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ E,
                                const int32_t* __restrict__ mat, int n_materials, double* __restrict__ Eb,
                                int32_t* __restrict__ Mb)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = __ldg(perm + j);
        if (MCX_IN_BOUNDS(l >= 0 && l < n, BC_PERM, l)) {
            Eb[j] = __ldg(E + l);
            const int32_t m = __ldg(mat + l);
            Mb[j] = m >= 0 && m < n_materials ? m : -1;
        } else {
            Eb[j] = __longlong_as_double(0x7ff8000000000000LL);
            Mb[j] = -1;
        }
    }
}

}  // namespace

template <bool LIN, typename OutT>
static int launch_warp2_t(const Tables& t, int64_t n, const double* E, const int32_t* mat, const int32_t* perm,
                          OutT* out, int grid, cudaStream_t st, unsigned long long* work, bool inb)
{
    switch (t.n_ch) {
    case 1: k_xs_lookup_warp2<1, kFastUnroll, 1, OutT, LIN><<<grid, 256, 0, st>>>(t, n, E, mat, perm, out, work, inb); break;
    case 2: k_xs_lookup_warp2<1, kFastUnroll, 2, OutT, LIN><<<grid, 256, 0, st>>>(t, n, E, mat, perm, out, work, inb); break;
    case 3: k_xs_lookup_warp2<2, kFastUnroll, 3, OutT, LIN><<<grid, 256, 0, st>>>(t, n, E, mat, perm, out, work, inb); break;
    case 4: k_xs_lookup_warp2<2, kFastUnroll, 4, OutT, LIN><<<grid, 256, 0, st>>>(t, n, E, mat, perm, out, work, inb); break;
    case 5: k_xs_lookup_warp2<2, kFastUnroll, 5, OutT, LIN><<<grid, 256, 0, st>>>(t, n, E, mat, perm, out, work, inb); break;
    default: return -1;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <typename OutT>
static int launch_fast_t(const Tables& t, int64_t n, const double* E, const int32_t* mat, const int32_t* perm,
                         OutT* out, int grid, cudaStream_t st, unsigned long long* work, bool linear, bool inb)
{
    // one instantiation per channel count: no work on unused record slots
#if MCX_FAST_WARP
    if (perm && work)
        return linear ? launch_warp2_t<true>(t, n, E, mat, perm, out, grid, st, work, inb)
                      : launch_warp2_t<false>(t, n, E, mat, perm, out, grid, st, work, inb);
#endif
    if (inb) return -1;   // binned inputs: the chunk-claiming warp forms only
    switch (t.n_ch) {
    case 1: k_xs_lookup_fast<1, kFastUnroll, 1, OutT><<<grid, 256, 0, st>>>(t, n, E, mat, perm, out, work); break;
    case 2: k_xs_lookup_fast<1, kFastUnroll, 2, OutT><<<grid, 256, 0, st>>>(t, n, E, mat, perm, out, work); break;
    case 3: k_xs_lookup_fast<2, kFastUnroll, 3, OutT><<<grid, 256, 0, st>>>(t, n, E, mat, perm, out, work); break;
    case 4: k_xs_lookup_fast<2, kFastUnroll, 4, OutT><<<grid, 256, 0, st>>>(t, n, E, mat, perm, out, work); break;
    case 5: k_xs_lookup_fast<2, kFastUnroll, 5, OutT><<<grid, 256, 0, st>>>(t, n, E, mat, perm, out, work); break;
    default: return -1;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_xs_lookup_fast(const Tables& t, int64_t n, const double* E, const int32_t* mat,
                          const int32_t* perm, void* out, bool out32, int grid, cudaStream_t st,
                          unsigned long long* work, bool linear, bool inputs_binned)
{
    if (work && cudaMemsetAsync(work, 0, sizeof(unsigned long long), st) != cudaSuccess) return -1;
    return out32 ? launch_fast_t(t, n, E, mat, perm, static_cast<float*>(out), grid, st, work, linear, inputs_binned)
                 : launch_fast_t(t, n, E, mat, perm, static_cast<double*>(out), grid, st, work, linear,
                                 inputs_binned);
}

template <int W, int NC, typename OutT>
static int launch_staged_nc(const Tables& t, const SortParams& sp, int64_t n, const double* E, const int32_t* mat,
                            const int32_t* perm, OutT* out, int grid, cudaStream_t st, unsigned long long* work,
                            unsigned int* err)
{
    const size_t smem = kStStages * StageLayout<W>::kBytes + 128;
    if (cudaFuncSetAttribute(k_xs_lookup_staged<W, kFastUnroll, NC, OutT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -1;
    // MCX_TEST_STAGED_STALL=1 (a test hook): the producers leave their first
    // chunk unstaged and every wait is limited to about 0.1 ms, so the
    // consumers' bounded waits run out and report through *err
    const char* hook = std::getenv("MCX_TEST_STAGED_STALL");
    const int stall = hook && hook[0] == '1' ? 1 : 0;
    const long long wait_cycles = stall ? 200000LL : kStWaitCycles;
    k_xs_lookup_staged<W, kFastUnroll, NC, OutT><<<grid, kStThreads, smem, st>>>(t, sp, n, E, mat, perm, out, work,
                                                                                 err, wait_cycles, stall);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <typename OutT>
static int launch_staged_t(const Tables& t, const SortParams& sp, int64_t n, const double* E, const int32_t* mat,
                           const int32_t* perm, OutT* out, int grid, cudaStream_t st, unsigned long long* work,
                           unsigned int* err)
{
    switch (t.n_ch) {
    case 1: return launch_staged_nc<1, 1>(t, sp, n, E, mat, perm, out, grid, st, work, err);
    case 2: return launch_staged_nc<1, 2>(t, sp, n, E, mat, perm, out, grid, st, work, err);
    case 3: return launch_staged_nc<2, 3>(t, sp, n, E, mat, perm, out, grid, st, work, err);
    case 4: return launch_staged_nc<2, 4>(t, sp, n, E, mat, perm, out, grid, st, work, err);
    case 5: return launch_staged_nc<2, 5>(t, sp, n, E, mat, perm, out, grid, st, work, err);
    default: return -1;
    }
}

int launch_xs_lookup_staged(const Tables& t, const SortParams& sp, int64_t n, const double* E,
                            const int32_t* mat, const int32_t* perm, void* out, bool out32, int sm_count,
                            cudaStream_t st, unsigned long long* work, unsigned int* err)
{
    const int grid = sm_count * MCX_STAGED_BLOCKS;
    if (!perm || !work || !err) return -1;
    if (t.max_mat_species > kStMaxSpecies || t.H == 0) return -2;   // the caller uses the global-memory form
    if (cudaMemsetAsync(work, 0, sizeof(unsigned long long), st) != cudaSuccess) return -1;
    return out32 ? launch_staged_t(t, sp, n, E, mat, perm, static_cast<float*>(out), grid, st, work, err)
                 : launch_staged_t(t, sp, n, E, mat, perm, static_cast<double*>(out), grid, st, work, err);
}

// Exclusive scan of bins[0, nb) (part sums at bins + nb + 1): parts of
// whole 1024-bin steps, at most kSortScanParts of them.
static void launch_bin_scan(uint32_t* bins, int nb, cudaStream_t st)
{
    int seg = (nb + kSortScanParts - 1) / kSortScanParts;
    seg = (seg + 1023) / 1024 * 1024;
    const int parts = (nb + seg - 1) / seg;
    uint32_t* part = bins + nb + 1;
    k_scan_part_sums<<<parts, 1024, 0, st>>>(bins, nb, seg, part);
    k_scan_parts<<<parts, 1024, 0, st>>>(bins, nb, seg, part);
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
    launch_bin_scan(bins, nb, st);
    k_lookup_sort_scatter<<<grid, 256, 0, st>>>(sp, n, E, mat, bins, perm);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

namespace {
struct Bin2Plan {
    int n_coarse, n_tiles;
    int64_t cells;   // n_coarse x n_tiles
};
Bin2Plan bin2_plan(const SortParams& sp, int64_t n)
{
    Bin2Plan b;
    const int64_t nbins = (int64_t)sp.n_materials * sp.n_ebuckets;
    b.n_coarse = (int)((nbins + (1 << kBinFineBits) - 1) >> kBinFineBits);
    b.n_tiles = (int)((n + kBinTile - 1) / kBinTile);
    b.cells = (int64_t)b.n_coarse * b.n_tiles;
    return b;
}
}  // namespace

size_t lookup_sort2_place_words(const SortParams& sp, int64_t n)
{
    return (size_t)bin2_plan(sp, n).cells + 1 + kSortScanParts;
}

int launch_lookup_sort2(const SortParams& sp, int64_t n, const double* E, const int32_t* mat, uint32_t* place,
                        uint32_t* keys, int32_t* tidx, uint16_t* tfine, int32_t* perm, int sm_count,
                        cudaStream_t st, const Bin2Carry* carry)
{
    const Bin2Plan b = bin2_plan(sp, n);
    // the tile scan covers 4 coarse bins per thread of pass A
    if (n < 1 || b.cells > ((int64_t)1 << 28) || b.n_coarse > 4 * kBin2Threads) return -2;
    const bool cy = carry != nullptr;
    const size_t smem = sizeof(uint32_t) * (size_t)b.n_coarse;
    // pass A: counts and starts, staged indices, staged keys (or with the
    // carry staged energies); pass B: counts and starts, staged indices and
    // fine bins (and with the carry energies)
    const size_t smem_a = sizeof(uint32_t) * (2 * (size_t)b.n_coarse + kBinTile) +
                          (cy ? sizeof(double) : sizeof(uint32_t)) * kBinTile;
    const size_t sub_b = cy ? Bin2Fine<true>::kSub : Bin2Fine<false>::kSub;
    const size_t smem_b = sizeof(uint32_t) * 2 * kBin2FineThreads + (sizeof(int32_t) + sizeof(uint16_t)) * sub_b +
                          (cy ? sizeof(double) * sub_b : 0);
    const void* ka = cy ? (const void*)k_bin2_scatter<true> : (const void*)k_bin2_scatter<false>;
    const void* kb = cy ? (const void*)k_bin2_fine<true> : (const void*)k_bin2_fine<false>;
    if (cudaFuncSetAttribute(ka, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_a) != cudaSuccess ||
        cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b) != cudaSuccess)
        return -1;
    const int g = b.n_tiles < sm_count * 4 ? b.n_tiles : sm_count * 4;
    k_bin2_count<<<g, 512, smem, st>>>(sp, n, E, mat, b.n_coarse, b.n_tiles, place, keys);
    launch_bin_scan(place, (int)b.cells, st);
    const int ga = b.n_tiles < sm_count * MCX_BIN2_A_BLOCKS ? b.n_tiles : sm_count * MCX_BIN2_A_BLOCKS;
    const int bpb = cy ? Bin2Fine<true>::kBlocks : Bin2Fine<false>::kBlocks;
    const int gb = b.n_coarse < sm_count * bpb ? b.n_coarse : sm_count * bpb;
    if (cy) {
        k_bin2_scatter<true><<<ga, kBin2Threads, smem_a, st>>>(n, keys, b.n_coarse, b.n_tiles, place, tidx, tfine, E,
                                                               carry->tE);
        k_bin2_fine<true><<<gb, Bin2Fine<true>::kThreads, smem_b, st>>>(n, b.n_coarse, b.n_tiles, place, tidx, tfine, perm,
                                                                carry->tE, sp.n_ebuckets, carry->Eb, carry->Mb);
    } else {
        k_bin2_scatter<false><<<ga, kBin2Threads, smem_a, st>>>(n, keys, b.n_coarse, b.n_tiles, place, tidx, tfine,
                                                                nullptr, nullptr);
        k_bin2_fine<false><<<gb, Bin2Fine<false>::kThreads, smem_b, st>>>(n, b.n_coarse, b.n_tiles, place, tidx, tfine, perm,
                                                                 nullptr, sp.n_ebuckets, nullptr, nullptr);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_gather_inputs(int64_t n, const int32_t* perm, const double* E, const int32_t* mat, int n_materials,
                         double* Eb, int32_t* Mb, int grid, cudaStream_t st)
{
    if (n < 1) return 0;
    k_gather_inputs<<<grid, 256, 0, st>>>(n, perm, E, mat, n_materials, Eb, Mb);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

MCX_BOUNDS_READER(bounds_error_xs_fast)

}  // namespace mcx
