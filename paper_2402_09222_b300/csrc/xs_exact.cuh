// xs_exact.cuh -- FP64 interpolation evaluated exactly as the plain
// definition is written (include only from translation units compiled with
// --fmad=false).
//
// Per species i of a material (Sec. 5.1, the macroscopic lookup): grid index
// k_i, fraction f = (E - g[k]) / (g[k+1] - g[k]) clamped to [0, 1], channel
// value sigma = s[k] + f * (s[k+1] - s[k]); sums run over the species in
// stored order starting from +0.0.
#pragma once

#include "mcx_internal.cuh"

namespace mcx {

__device__ __forceinline__ double fraction_exact(double E, double g0, double g1)
{
    double f = (E - g0) / (g1 - g0);
    if (f < 0.0) f = 0.0;
    if (f > 1.0) f = 1.0;
    return f;
}

__device__ __forceinline__ double interp_exact(double s0, double s1, double f)
{
    return s0 + f * (s1 - s0);
}

// Transport lookup: Sigma_t = sum_i N_i (sigma_s,i + sigma_a,i) and
// Sigma_a = sum_i N_i sigma_a,i, both sequential in species order.  The
// running sums C_i of Sigma_t are stored to cum[0..n-1] (the collision picks
// its species from them).
template <typename T>
__device__ __forceinline__ void macro_transport(const Tables& t, int32_t m, double E,
                                                double& sig_t, double& sig_a, double* cum)
{
    const int64_t eb = search_key(E);
    const int32_t hb = t.H > 0 ? hash_bin(t, E, eb) : 0;
    const int32_t i0 = __ldg(t.moff + m), i1 = __ldg(t.moff + m + 1);
    const int32_t nc = t.n_ch, cs = t.ch_scatter, ca = t.ch_absorb;
    double st = 0.0, sa = 0.0;
    for (int32_t i = i0; i < i1; ++i) {
        const int32_t s = __ldg(t.msp + i);
        const double N = __ldg(t.mden + i);
        const int64_t k = species_index(t, s, eb, hb);
        const int64_t p = __ldg(t.goff + s) + k;
        const double f = fraction_exact(E, __ldg(t.E + p), __ldg(t.E + p + 1));
        const double ss = interp_exact(sig_at<T>(t.sigma, p * nc + cs),
                                       sig_at<T>(t.sigma, (p + 1) * nc + cs), f);
        const double sai = interp_exact(sig_at<T>(t.sigma, p * nc + ca),
                                        sig_at<T>(t.sigma, (p + 1) * nc + ca), f);
        st = st + N * (ss + sai);
        sa = sa + N * sai;
        cum[i - i0] = st;
    }
    sig_t = st;
    sig_a = sa;
}

}  // namespace mcx
