// xs_exact.cuh -- FP64 interpolation evaluated exactly as the plain
// definition is written (include only from translation units compiled with
// --fmad=false), and the transport lookup, which differs from it only in the
// last bits (see MCX_TRANSPORT_RECIP below).
//
// Per species i of a material (Sec. 5.1, the macroscopic lookup): grid index
// k_i, fraction f = (E - g[k]) / (g[k+1] - g[k]) clamped to [0, 1], channel
// value sigma = s[k] + f * (s[k+1] - s[k]); sums run over the species in
// stored order starting from +0.0.
#pragma once

#include "mcx_internal.cuh"

namespace mcx {

// The clamps compare bit patterns on the integer pipes (f is never NaN here:
// callers handle NaN energies before; a -0.0 clamped to +0.0 changes no
// result because it only multiplies a finite difference added to s[k]).
__device__ __forceinline__ double fraction_exact(double E, double g0, double g1)
{
    double f = (E - g0) / (g1 - g0);
    const int64_t fb = __double_as_longlong(f);
    if (fb < 0) f = 0.0;
    if (fb > 0x3FF0000000000000LL) f = 1.0;
    return f;
}

// The transport lookup departs from the as-written FP64 evaluation in ways
// that cost it at most an ulp or two per value, because the FP64 pipe (1/64
// of the FP32 rate on B300) bounds the event kernels:
//  - the fraction multiplies by a stored reciprocal interval width instead
//    of dividing (one multiply instead of a multi-instruction division);
//  - the interpolation s0 + f (s1 - s0) is one fused multiply-add;
//  - inside a grid, s0 + (E - g0) slope with the slope stored per interval,
//    the total s_scatter + s_absorb interpolated from stored per-point totals,
//    and the density folded into the running sums (Sigma += N sigma as one
//    fused multiply-add): 5 FP64 operations per species instead of 10.
// Measured on the 17x17 lattice: 7.50e6 -> 8.74e6 -> 9.27e6 particles/s for
// the first two, 9.8e6 -> 1.05e7 for the stored slopes, -> 1.11e7 for the
// stored totals and the folded densities.
// A decision (flight length against a surface, the collision's species and
// reaction) could only change if a random number fell within that last-bit
// difference of its threshold; every history-matched test still reproduces
// the per-history collision counts exactly.  The standalone lookup entry
// points keep the exact definition (fraction_exact, interp_exact).
#ifndef MCX_TRANSPORT_RECIP
#define MCX_TRANSPORT_RECIP 1
#endif
#ifndef MCX_TRANSPORT_FMA
#define MCX_TRANSPORT_FMA 1
#endif
__device__ __forceinline__ double fraction_transport(const Tables& t, double E, int64_t p)
{
#if MCX_TRANSPORT_RECIP
    double f = (E - __ldg(t.E + p)) * __ldg(t.winv + p);
    const int64_t fb = __double_as_longlong(f);
    if (fb < 0) f = 0.0;
    if (fb > 0x3FF0000000000000LL) f = 1.0;
    return f;
#else
    return fraction_exact(E, __ldg(t.E + p), __ldg(t.E + p + 1));
#endif
}

__device__ __forceinline__ double interp_exact(double s0, double s1, double f)
{
    return s0 + f * (s1 - s0);
}

__device__ __forceinline__ double interp_transport(double s0, double s1, double f)
{
#if MCX_TRANSPORT_FMA
    return fma(f, s1 - s0, s0);
#else
    return s0 + f * (s1 - s0);
#endif
}

// Transport value of channel ch of the interval starting at point p, for an
// energy with g[p] <= E < g[p+1] (or E below the grid at a species' first
// point): s[p] + (E - g[p]) * slope[p] with the slope stored per interval --
// one fused multiply-add per channel instead of a subtraction and one, and no
// fraction (its multiply and clamps) -- a difference in the last bits from
// s[p] + f (s[p+1] - s[p]), like the reciprocal width above.  d < 0 (below
// the grid) clamps to 0, giving s[p] as the clamped fraction does.  The last
// interval of a species, where E may lie above the grid, keeps the fraction
// form and its clamp to 1.
#ifndef MCX_TRANSPORT_SLOPE
#define MCX_TRANSPORT_SLOPE 1
#endif
__device__ __forceinline__ double offset_transport(const Tables& t, double E, int64_t p)
{
    double d = E - __ldg(t.E + p);
    if (__double_as_longlong(d) < 0) d = 0.0;
    return d;
}

template <typename T>
__device__ __forceinline__ double slope_value(const Tables& t, double d, int64_t p, int nc, int ch)
{
    return fma(d, __ldg(t.slope + p * nc + ch), sig_at<T>(t.sigma, p * nc + ch));
}

template <typename T>
__device__ __forceinline__ double fraction_value(const Tables& t, double f, int64_t p, int nc, int ch)
{
    return interp_transport(sig_at<T>(t.sigma, p * nc + ch), sig_at<T>(t.sigma, (p + 1) * nc + ch), f);
}

// Total (scatter + absorption) and absorption (and with NF nu-fission)
// cross sections of one species at E, its interval starting at point p,
// `last` its last interval.  Inside the grid the total comes from the stored
// per-point totals and their slopes (one fused multiply-add).
template <typename T, bool NF>
__device__ __forceinline__ void species_transport(const Tables& t, double E, int64_t p, int64_t last, double& stot,
                                                  double& sa, double& sf)
{
    const int nc = t.n_ch, cs = t.ch_scatter, ca = t.ch_absorb, cf = t.ch_nu_fission;
#if MCX_TRANSPORT_SLOPE
    if (p < last) {
        const double d = offset_transport(t, E, p);
        const double2 tt = __ldg(t.ttot + p);
        stot = fma(d, tt.y, tt.x);
        sa = slope_value<T>(t, d, p, nc, ca);
        if (NF) sf = slope_value<T>(t, d, p, nc, cf);
        return;
    }
#endif
    const double f = fraction_transport(t, E, p);
    sa = fraction_value<T>(t, f, p, nc, ca);
    stot = fraction_value<T>(t, f, p, nc, cs) + sa;
    if (NF) sf = fraction_value<T>(t, f, p, nc, cf);
}

// Transport lookup: Sigma_t = sum_i N_i (sigma_s,i + sigma_a,i) and
// Sigma_a = sum_i N_i sigma_a,i, both sequential in species order.  The
// running sums C_i of Sigma_t are stored to cum[0..n-1] (the collision picks
// its species from them).  MCX_TRANSPORT_INFLIGHT species are evaluated at a
// time so their load chains overlap; their terms are still added one after
// the other, in species order, so every sum is the sequential FP64 value.  With NF the nu-fission
// sum nuSigma_f = sum_i N_i nu sigma_f,i is formed the same way.
// Species whose load chains (entry, hash window, search probes, records) are
// in flight together per thread.  With FP64 sums 2 measured fastest on the
// 17x17 lattice (886 ms per 1e7 histories; 3: 906, 4: 905); with the FP32-pair
// sums below, which leave the FP64 pipe, 4 (652 ms; 2: 665, 3: 665).
#ifndef MCX_CUM_VEC
#define MCX_CUM_VEC 1
#endif
#ifndef MCX_TRANSPORT_INFLIGHT
#define MCX_TRANSPORT_INFLIGHT 4
#endif
template <typename T, bool NF = false>
__device__ __forceinline__ void macro_transport(const Tables& t, int32_t m, double E,
                                                double& sig_t, double& sig_a, double* cum,
                                                double* sig_nf = nullptr)
{
    const int64_t eb = search_key(E);
    const int32_t hb = t.H > 0 ? hash_bin(t, E, eb) : 0;
    const int32_t i0 = __ldg(t.moff + m), i1 = __ldg(t.moff + m + 1);
    constexpr int TU = MCX_TRANSPORT_INFLIGHT;
    double st = 0.0, sa = 0.0, nf = 0.0;
    for (int32_t i = i0; i < i1; i += TU) {
        int32_t base[TU], len[TU], last[TU];
        double N[TU];
#pragma unroll
        for (int u = 0; u < TU; ++u) {
            const int32_t ii = i + u < i1 ? i + u : i1 - 1;
            N[u] = __ldg(t.mden + ii);
            const int4 e = __ldg(t.ment + ii);
            last[u] = e.x + e.y - 2;
            search_window(t, e, hb, base[u], len[u]);
        }
        for (int s = 0; s < t.search_steps; ++s) {
#pragma unroll
            for (int u = 0; u < TU; ++u) search_step(t.E, base[u], len[u], eb);
        }
        double c[TU], a[TU], v[TU];
#pragma unroll
        for (int u = 0; u < TU; ++u) {
            v[u] = 0.0;
            species_transport<T, NF>(t, E, base[u], last[u], c[u], a[u], v[u]);
        }
        // density folded into the running sums: one fused multiply-add each,
        // in species order
#pragma unroll
        for (int u = 0; u < TU; ++u) {
            if (u == 0 || i + u < i1) {
                st = fma(N[u], c[u], st);
                sa = fma(N[u], a[u], sa);
                if (NF) nf = fma(N[u], v[u], nf);
                cum[i + u - i0] = st;
            }
        }
    }
    sig_t = st;
    sig_a = sa;
    if (NF) *sig_nf = nf;
}

// macro_transport for one particle on a whole converged warp, for when few
// particles need a lookup (the tail of an event loop, where one thread's
// chain of dependent loads over a material's species is the latency of the
// whole iteration): lane s evaluates species i0 + s, i0 + 32 + s, ... (all
// their load chains in flight at once), then every lane adds the terms in
// species order with the same fused multiply-adds -- bit-identical to
// macro_transport; lane 0 stores the running sums.
template <typename T, bool NF = false>
__device__ __forceinline__ void macro_transport_warp(const Tables& t, int32_t m, double E, double& sig_t,
                                                     double& sig_a, double* cum, double* sig_nf = nullptr)
{
    const int lane = threadIdx.x & 31;
    const int64_t eb = search_key(E);
    const int32_t hb = t.H > 0 ? hash_bin(t, E, eb) : 0;
    const int32_t i0 = __ldg(t.moff + m), i1 = __ldg(t.moff + m + 1);
    double st = 0.0, sa = 0.0, nf = 0.0;
    for (int32_t i = i0; i < i1; i += 32) {
        const int32_t ii = i + lane;
        double N = 0.0, c = 0.0, a = 0.0, v = 0.0;
        if (ii < i1) {
            N = __ldg(t.mden + ii);
            const int4 e = __ldg(t.ment + ii);
            int32_t base, len;
            search_window(t, e, hb, base, len);
            for (int s = 0; s < t.search_steps; ++s) search_step(t.E, base, len, eb);
            species_transport<T, NF>(t, E, base, e.x + e.y - 2, c, a, v);
        }
        const int n = i1 - i < 32 ? i1 - i : 32;
        for (int s = 0; s < n; ++s) {
            const double Ns = __shfl_sync(0xffffffffu, N, s);
            st = fma(Ns, __shfl_sync(0xffffffffu, c, s), st);
            sa = fma(Ns, __shfl_sync(0xffffffffu, a, s), sa);
            if (NF) nf = fma(Ns, __shfl_sync(0xffffffffu, v, s), nf);
            if (lane == 0) cum[i + s - i0] = st;
        }
    }
    sig_t = st;
    sig_a = sa;
    if (NF) *sig_nf = nf;
}

// ---------------------------------------------------------------------------
// The transport lookup in FP32 pairs ("double-float": a value is (hi, lo)
// with hi = RN(hi + lo)).  Knuth's TwoSum gives a sum's rounding error
// exactly and a fused multiply-add a product's, so a + b c comes out within
// a few 2^-48 of |a| + |b c| -- about 2^-44 relative where a and b c do not
// cancel -- using FP32 operations only, which B300 runs at 64 times its
// FP64 rate.  Energies, the grid search (FP64 bit patterns) and every tally
// stay FP64; Sigma_t, Sigma_a (and nuSigma_f) and the running sums C_i carry
// ~1e-12 relative against the FP64 sums, so a decision (a flight against a
// surface, the species of a collision) changes only if a random number falls
// that close to its threshold.  The collision re-evaluates its chosen
// species in FP64 (species_transport).
#ifndef MCX_TRANSPORT_PAIRS
#define MCX_TRANSPORT_PAIRS 1
#endif

__device__ __forceinline__ float2 pair_two_sum(float a, float b)
{
    const float s = a + b;
    const float bp = s - a;
    return make_float2(s, (a - (s - bp)) + (b - bp));
}

// a - b
__device__ __forceinline__ float2 pair_sub(float2 a, float2 b)
{
    const float2 s = pair_two_sum(a.x, -b.x);
    const float e = s.y + (a.y - b.y);
    const float h = s.x + e;
    return make_float2(h, e - (h - s.x));
}

// a + b c
__device__ __forceinline__ float2 pair_fma(float2 a, float2 b, float2 c)
{
    const float p = b.x * c.x;
    float pe = fmaf(b.x, c.x, -p);
    pe = fmaf(b.x, c.y, fmaf(b.y, c.x, pe));
    const float2 s = pair_two_sum(a.x, p);
    const float e = s.y + (a.y + pe);
    const float h = s.x + e;
    return make_float2(h, e - (h - s.x));
}

// Exact FP32 -> FP64 widening with integer operations for a finite value of
// either sign (a pair's low part may be negative); zero and subnormals take
// the conversion instruction.
__device__ __forceinline__ double widen_signed(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t m = u & 0x7FFFFFFFu;
    const uint32_t e = m >> 23;
    if (e == 0u) return (double)f;
    const uint32_t hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((m & 0x7FFFFFu) >> 3);
    return __hiloint2double((int)hi, (int)(u << 29));
}

// hi + lo in FP64 (one FP64 add)
__device__ __forceinline__ double pair_value(float2 v) { return widen_signed(v.x) + widen_signed(v.y); }

// E as a pair: hi = E rounded to FP32, lo = the rest
__device__ __forceinline__ float2 energy_pair(double E)
{
    const float h = (float)E;
    return make_float2(h, (float)(E - widen_signed(h)));
}

// Total, absorption (and with NF nu-fission) of one species at the energy
// pair Ep (key eb), its interval starting at point p, `last` its last
// interval: s[p] + (E - g[p]) slope[p] with E - g[p] clamped to [0, the
// interval] as the clamped fraction is.
template <bool NF>
__device__ __forceinline__ void species_pair(const Tables& t, float2 Ep, int64_t eb, int64_t p, int64_t last,
                                             float2& tot, float2& sa, float2& sf)
{
    const float4* q = t.tpair + p * t.tpair_w;
    const float4 q0 = __ldg(q), q1 = __ldg(q + 1), q2 = __ldg(q + 2);
    float2 Ex = Ep;
    if (p == last && eb >= ebits(__ldg(t.E + p + 1))) {   // at or above the grid's top
        const float4 qn = __ldg(q + t.tpair_w);
        Ex = make_float2(qn.x, qn.y);
    }
    float2 d = pair_sub(Ex, make_float2(q0.x, q0.y));
    if (d.x < 0.f) d = make_float2(0.f, 0.f);                // below the grid
    tot = pair_fma(make_float2(q0.z, q0.w), d, make_float2(q1.x, q1.y));
    sa = pair_fma(make_float2(q1.z, q1.w), d, make_float2(q2.x, q2.y));
    if (NF) {
        const float4 q3 = __ldg(q + 3);
        sf = pair_fma(make_float2(q2.z, q2.w), d, make_float2(q3.x, q3.y));
    }
}

// macro_transport in pairs: the same species, search and order; C_i stored
// as pairs (cum2) for the collision's comparison.
template <bool NF = false>
__device__ __forceinline__ void macro_transport_pair(const Tables& t, int32_t m, double E, double& sig_t,
                                                     double& sig_a, float2* cum2, double* sig_nf = nullptr)
{
    constexpr int TU = MCX_TRANSPORT_INFLIGHT;
    const int64_t eb = search_key(E);
    const int32_t hb = t.H > 0 ? hash_bin(t, E, eb) : 0;
    const float2 Ep = energy_pair(E);
    const int32_t i0 = __ldg(t.moff + m), i1 = __ldg(t.moff + m + 1);
    float2 st = make_float2(0.f, 0.f), sa = st, nf = st;
    for (int32_t i = i0; i < i1; i += TU) {
        int32_t base[TU], len[TU], last[TU];
        float2 N[TU];
#pragma unroll
        for (int u = 0; u < TU; ++u) {
            const int32_t ii = i + u < i1 ? i + u : i1 - 1;
            N[u] = __ldg(t.mden2 + ii);
            const int4 e = __ldg(t.ment + ii);
            last[u] = e.x + e.y - 2;
            search_window(t, e, hb, base[u], len[u]);
        }
        for (int s = 0; s < t.search_steps; ++s) {
#pragma unroll
            for (int u = 0; u < TU; ++u) search_step(t.E, base[u], len[u], eb);
        }
        float2 c[TU], a[TU], v[TU];
#pragma unroll
        for (int u = 0; u < TU; ++u) {
            v[u] = make_float2(0.f, 0.f);
            species_pair<NF>(t, Ep, eb, base[u], last[u], c[u], a[u], v[u]);
        }
#pragma unroll
        for (int u = 0; u < TU; ++u) {
            if (u == 0 || i + u < i1) {
                st = pair_fma(st, N[u], c[u]);
                sa = pair_fma(sa, N[u], a[u]);
                if (NF) nf = pair_fma(nf, N[u], v[u]);
#if MCX_CUM_VEC && MCX_TRANSPORT_INFLIGHT == 4
            }
            c[u] = st;   // C_{i+u}; past the last species it repeats the sum
        }
        // the group's four sums as two 16-byte stores: cum2 rows hold a
        // multiple of 4 entries and start 32-byte aligned, i - i0 is a
        // multiple of 4, and entries past the material's species are never read
        float4* row = reinterpret_cast<float4*>(cum2 + (i - i0));
        row[0] = make_float4(c[0].x, c[0].y, c[1].x, c[1].y);
        row[1] = make_float4(c[2].x, c[2].y, c[3].x, c[3].y);
#else
                cum2[i + u - i0] = st;
            }
        }
#endif
    }
    sig_t = pair_value(st);
    sig_a = pair_value(sa);
    if (NF) *sig_nf = pair_value(nf);
}

// macro_transport_pair on a whole converged warp (lanes over species, the
// sums in species order by every lane): the same values.
template <bool NF = false>
__device__ __forceinline__ void macro_transport_pair_warp(const Tables& t, int32_t m, double E, double& sig_t,
                                                          double& sig_a, float2* cum2, double* sig_nf = nullptr)
{
    const int lane = threadIdx.x & 31;
    const int64_t eb = search_key(E);
    const int32_t hb = t.H > 0 ? hash_bin(t, E, eb) : 0;
    const float2 Ep = energy_pair(E);
    const int32_t i0 = __ldg(t.moff + m), i1 = __ldg(t.moff + m + 1);
    float2 st = make_float2(0.f, 0.f), sa = st, nf = st;
    for (int32_t i = i0; i < i1; i += 32) {
        const int32_t ii = i + lane;
        float2 N = make_float2(0.f, 0.f), c = N, a = N, v = N;
        if (ii < i1) {
            N = __ldg(t.mden2 + ii);
            const int4 e = __ldg(t.ment + ii);
            int32_t base, len;
            search_window(t, e, hb, base, len);
            for (int s = 0; s < t.search_steps; ++s) search_step(t.E, base, len, eb);
            species_pair<NF>(t, Ep, eb, base, e.x + e.y - 2, c, a, v);
        }
        const int n = i1 - i < 32 ? i1 - i : 32;
        for (int s = 0; s < n; ++s) {
            const float2 Ns = make_float2(__shfl_sync(0xffffffffu, N.x, s), __shfl_sync(0xffffffffu, N.y, s));
            st = pair_fma(st, Ns, make_float2(__shfl_sync(0xffffffffu, c.x, s), __shfl_sync(0xffffffffu, c.y, s)));
            sa = pair_fma(sa, Ns, make_float2(__shfl_sync(0xffffffffu, a.x, s), __shfl_sync(0xffffffffu, a.y, s)));
            if (NF)
                nf = pair_fma(nf, Ns, make_float2(__shfl_sync(0xffffffffu, v.x, s), __shfl_sync(0xffffffffu, v.y, s)));
            if (lane == 0) cum2[i + s - i0] = st;
        }
    }
    sig_t = pair_value(st);
    sig_a = pair_value(sa);
    if (NF) *sig_nf = pair_value(nf);
}

}  // namespace mcx
