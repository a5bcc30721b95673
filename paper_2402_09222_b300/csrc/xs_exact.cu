// xs_exact.cu -- macroscopic lookup with the plain definition's FP64
// arithmetic (compiled with --fmad=false), the grid-index debug kernel and
// the hash-grid builder.
#include "xs_exact.cuh"
#include "kernels.h"

namespace mcx {

// One thread per lookup.  For lookup l: out[l][r] = sum_i N_i sigma_{r,i}(E).
// `perm` (optional) is a processing order: thread j handles lookup perm[j];
// results land at the lookup's own row, so the order changes nothing.
template <typename T>
__global__ void __launch_bounds__(256) k_xs_lookup_exact(Tables t, int64_t n,
                                                         const double* __restrict__ Ein,
                                                         const int32_t* __restrict__ mat,
                                                         const int32_t* __restrict__ perm,
                                                         double* __restrict__ out)
{
    const int nc = t.n_ch;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = perm ? (int64_t)__ldg(perm + j) : j;
        if (perm && !MCX_IN_BOUNDS(l >= 0 && l < n, BC_PERM, l)) continue;
        const double E = __ldg(Ein + l);
        const int32_t m = __ldg(mat + l);
        double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        if (m < 0 || m >= t.n_materials || E != E) {
            for (int r = 0; r < nc; ++r) out[l * nc + r] = __longlong_as_double(0x7ff8000000000000LL);
            continue;
        }
        const int64_t eb = search_key(E);
        const int32_t hb = t.H > 0 ? hash_bin(t, E, eb) : 0;
        const int32_t i0 = __ldg(t.moff + m), i1 = __ldg(t.moff + m + 1);
        for (int32_t i = i0; i < i1; ++i) {
            const int32_t s = __ldg(t.msp + i);
            const double N = __ldg(t.mden + i);
            const int64_t k = species_index(t, s, eb, hb);
            const int64_t p = __ldg(t.goff + s) + k;
            const double f = fraction_exact(E, __ldg(t.E + p), __ldg(t.E + p + 1));
#pragma unroll
            for (int r = 0; r < 5; ++r) {
                if (r < nc) {
                    const double sg = interp_exact(sig_at<T>(t.sigma, p * nc + r),
                                                   sig_at<T>(t.sigma, (p + 1) * nc + r), f);
                    acc[r] = acc[r] + N * sg;
                }
            }
        }
#pragma unroll
        for (int r = 0; r < 5; ++r)
            if (r < nc) out[l * nc + r] = acc[r];
    }
}

__global__ void k_xs_indices(Tables t, int64_t n, const double* __restrict__ Ein,
                             const int32_t* __restrict__ mat, int32_t max_species,
                             int32_t* __restrict__ kout)
{
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
         l += (int64_t)gridDim.x * blockDim.x) {
        const double E = Ein[l];
        const int32_t m = mat[l];
        const bool ok = m >= 0 && m < t.n_materials;
        const int32_t i0 = ok ? t.moff[m] : 0, cnt = ok ? t.moff[m + 1] - i0 : 0;
        const int64_t eb = search_key(E);
        const int32_t hb = t.H > 0 ? hash_bin(t, E, eb) : 0;
        for (int32_t i = 0; i < max_species; ++i)
            kout[l * max_species + i] =
                i < cnt ? (int32_t)species_index(t, t.msp[i0 + i], eb, hb) : -1;
    }
}

// hidx[s][b] = largest k in [0, n_s-2] with g_s[k] <= hbound[b] (full search).
__global__ void k_build_hash(Tables t, int32_t* __restrict__ hidx)
{
    const int64_t total = (int64_t)t.n_species * (t.H + 1);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = (int32_t)(q / (t.H + 1));
        const int32_t b = (int32_t)(q % (t.H + 1));
        const int64_t base = t.goff[s], n = t.goff[s + 1] - base;
        hidx[q] = (int32_t)bsearch_window(t.E + base, 0, n - 2, ebits(t.hbound[b]));
    }
}

__global__ void k_hash_max_window(Tables t, int32_t* __restrict__ out)
{
    const int64_t total = (int64_t)t.n_species * t.H;
    int32_t best = 1;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = q / t.H, b = q % t.H;
        const int32_t* h = t.hidx + s * (t.H + 1) + b;
        const int32_t w = h[1] - h[0] + 1;
        best = w > best ? w : best;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const int32_t v = __shfl_xor_sync(0xffffffffu, best, o);
        best = v > best ? v : best;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

int launch_hash_max_window(const Tables& t, int32_t* out, int grid, cudaStream_t st)
{
    k_hash_max_window<<<grid, 256, 0, st>>>(t, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Copy new densities and cross sections from device buffers into the exact
// tables (sigma rounded to the table precision) and into the fast path's
// copies (the FP32 density in each material entry, the FP32 point records).
__global__ void k_update_tables(Tables t, const double* __restrict__ dens_src, int64_t nnz,
                                double* __restrict__ mden, int4* __restrict__ ment,
                                const double* __restrict__ sig_src, void* __restrict__ sigma,
                                float4* __restrict__ frec)
{
    const int64_t n_sig = sig_src ? t.n_points * t.n_ch : 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz || i < n_sig; i += stride) {
        if (dens_src && i < nnz) {
            mden[i] = dens_src[i];
            ment[i].w = __float_as_int((float)dens_src[i]);
        }
        if (i < n_sig) {
            if (t.precision == MCX_FP32) static_cast<float*>(sigma)[i] = (float)sig_src[i];
            else static_cast<double*>(sigma)[i] = sig_src[i];
            const int64_t pt = i / t.n_ch, r = i % t.n_ch;
            reinterpret_cast<float*>(frec)[pt * 4 * t.frec_w + 2 + r] = (float)sig_src[i];
        }
    }
}

template <typename T>
__global__ void k_build_slopes(Tables t, double* __restrict__ slope)
{
    const int64_t n = t.n_points * t.n_ch;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t p = i / t.n_ch;
        // winv is 0 exactly at a species' last point, which starts no interval
        double v = 0.0;
        if (t.winv[p] != 0.0)
            v = (sig_at<T>(t.sigma, i + t.n_ch) - sig_at<T>(t.sigma, i)) / (t.E[p + 1] - t.E[p]);
        slope[i] = v;
    }
}

template <typename T>
__device__ __forceinline__ double total_at(const Tables& t, int64_t p)
{
    return sig_at<T>(t.sigma, p * t.n_ch + t.ch_scatter) + sig_at<T>(t.sigma, p * t.n_ch + t.ch_absorb);
}

template <typename T>
__global__ void k_build_totals(Tables t, double2* __restrict__ ttot)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < t.n_points; p += stride) {
        const double s0 = total_at<T>(t, p);
        double v = 0.0;
        if (t.winv[p] != 0.0) v = (total_at<T>(t, p + 1) - s0) / (t.E[p + 1] - t.E[p]);
        ttot[p] = make_double2(s0, v);
    }
}

int launch_build_slopes(const Tables& t, double* slope, double2* ttot, int grid, cudaStream_t st)
{
    const bool tr = t.ch_scatter >= 0 && t.ch_scatter < t.n_ch && t.ch_absorb >= 0 && t.ch_absorb < t.n_ch;
    if (t.precision == MCX_FP32) {
        k_build_slopes<float><<<grid, 256, 0, st>>>(t, slope);
        if (tr) k_build_totals<float><<<grid, 256, 0, st>>>(t, ttot);
    } else {
        k_build_slopes<double><<<grid, 256, 0, st>>>(t, slope);
        if (tr) k_build_totals<double><<<grid, 256, 0, st>>>(t, ttot);
    }
    if (!tr && cudaMemsetAsync(ttot, 0, sizeof(double2) * (size_t)t.n_points, st) != cudaSuccess) return -1;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// x as an FP32 pair: hi = x rounded to FP32, lo = the rest rounded to FP32.
__device__ __forceinline__ float2 split_pair(double x)
{
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
}

template <typename T>
__global__ void k_build_pairs(Tables t, float4* __restrict__ tpair, float2* __restrict__ mden2, int64_t nnz)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int nc = t.n_ch, ca = t.ch_absorb, cf = t.ch_nu_fission;
    const bool tr = t.ch_scatter >= 0 && t.ch_scatter < nc && ca >= 0 && ca < nc;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < t.n_points; p += stride) {
        const float2 g = split_pair(t.E[p]);
        float2 tot = make_float2(0.f, 0.f), slt = tot, sa = tot, sla = tot, sf = tot, slf = tot;
        if (tr) {
            tot = split_pair(t.ttot[p].x);
            slt = split_pair(t.ttot[p].y);
            sa = split_pair(sig_at<T>(t.sigma, p * nc + ca));
            sla = split_pair(t.slope[p * nc + ca]);
            if (cf >= 0 && cf < nc) {
                sf = split_pair(sig_at<T>(t.sigma, p * nc + cf));
                slf = split_pair(t.slope[p * nc + cf]);
            }
        }
        float4* q = tpair + p * t.tpair_w;
        q[0] = make_float4(g.x, g.y, tot.x, tot.y);
        q[1] = make_float4(slt.x, slt.y, sa.x, sa.y);
        q[2] = make_float4(sla.x, sla.y, sf.x, sf.y);
        if (t.tpair_w > 3) q[3] = make_float4(slf.x, slf.y, 0.f, 0.f);
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += stride)
        mden2[i] = split_pair(t.mden[i]);
}

int launch_build_pairs(const Tables& t, float4* tpair, float2* mden2, int64_t nnz, int grid, cudaStream_t st)
{
    if (t.precision == MCX_FP32) k_build_pairs<float><<<grid, 256, 0, st>>>(t, tpair, mden2, nnz);
    else k_build_pairs<double><<<grid, 256, 0, st>>>(t, tpair, mden2, nnz);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_update_tables(const Tables& t, const double* dens_src, int64_t nnz, double* mden,
                         int4* ment, const double* sig_src, void* sigma, float4* frec,
                         cudaStream_t st)
{
    const int64_t n_sig = sig_src ? t.n_points * t.n_ch : 0;
    const int64_t n = nnz > n_sig ? nnz : n_sig;
    int grid = (int)((n + 255) / 256);
    if (grid > 4096) grid = 4096;
    if (grid < 1) grid = 1;
    k_update_tables<<<grid, 256, 0, st>>>(t, dens_src, nnz, mden, ment, sig_src, sigma, frec);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_xs_lookup_exact(const Tables& t, int64_t n, const double* E, const int32_t* mat,
                           const int32_t* perm, double* out, int grid, cudaStream_t st)
{
    if (t.precision == MCX_FP32)
        k_xs_lookup_exact<float><<<grid, 256, 0, st>>>(t, n, E, mat, perm, out);
    else
        k_xs_lookup_exact<double><<<grid, 256, 0, st>>>(t, n, E, mat, perm, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_xs_indices(const Tables& t, int64_t n, const double* E, const int32_t* mat,
                      int32_t max_species, int32_t* kout, int grid, cudaStream_t st)
{
    k_xs_indices<<<grid, 256, 0, st>>>(t, n, E, mat, max_species, kout);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_build_hash(const Tables& t, int32_t* hidx, int grid, cudaStream_t st)
{
    k_build_hash<<<grid, 256, 0, st>>>(t, hidx);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

MCX_BOUNDS_READER(bounds_error_xs_exact)

}  // namespace mcx
