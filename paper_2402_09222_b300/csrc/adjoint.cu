// adjoint.cu -- backward pass of the macroscopic lookup (compiled with
// --fmad=false).  The lookup is linear in the densities N_j and in the table
// entries s[k], s[k+1]:  Sigma_r = sum_j N_j ((1 - f) s_r[k] + f s_r[k+1]),
// so for a cotangent g_r of the output
//   dL/dN_j       = sum_r g_r sigma_{r,j}(E)
//   dL/ds_r[k]   += N_j (1 - f) g_r,     dL/ds_r[k+1] += N_j f g_r.
//
// The lookups are taken in the binned order (material, log-energy bucket),
// 32 at a time per warp.  A warp whose 32 lookups share one material sorts
// them by energy (a bitonic network over the lanes) and then turns its lanes
// over to the material's species, one species per lane.  For species j the
// sorted lookups fall into a few consecutive grid intervals q (usually one),
// each holding a contiguous run of lanes; per run the two sums
//   A_r = sum_l (1 - f_l) g_lr,   B_r = sum_l f_l g_lr
// give all of that run's contributions: one FP64 atomic per channel and
// point (dL/ds_r[q] += N_j A_r, dL/ds_r[q+1] += N_j B_r, instead of one per
// lookup), and dL/dN_j += sum_r (A_r s_r[q] + B_r s_r[q+1]), summed per lane
// and then per block in shared memory before one atomic per entry.
// Within a run in interval [g0, g1], f_l = (d_l + delta0) w with d_l =
// E_l - E_ref (E_ref the warp's lowest energy), delta0 = E_ref - g0 and
// w = 1 / (g1 - g0), so
//   B_r = w (S_r + delta0 G_r),   A_r = w (delta1 G_r - S_r)
// with G_r = sum_l g_lr and S_r = sum_l d_l g_lr over the run, taken as
// differences of prefix sums over the sorted lanes (formed once per warp for
// all species), and delta1 = g1 - E_ref.  While the warp's energy span is at
// most a few interval widths every term is bounded by the interval's width,
// so the rounding stays at a few ulps of sum_l |g_lr|, as in a sequential
// sum; a warp spread wider (sparse lookups) sums its runs lookup by lookup
// from shared memory instead.  Energies below a grid (f = 0) and at or above
// its top (f = 1) add their runs' G_r to one side.  Warps that mix
// materials, or hold an invalid lookup or the ragged tail, take the
// per-lookup form with one atomic per contribution.
//
// This moves the FP64 work (B300 runs FP64 at 1/64 of its FP32 rate) from
// per lookup and species to per warp and species, and the atomics likewise.
#include "kernels.h"
#include "xs_exact.cuh"

namespace mcx {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kBwThreads = 256;
constexpr int kBwWarps = kBwThreads / 32;
constexpr int kBwChunk = 128;          // lookups a warp claims at a time
constexpr int kBwMaxCh = 5;

// One lookup, every species, one atomic per contribution.
template <typename T>
__device__ __forceinline__ void backward_one(const Tables& t, int64_t l, double E, int32_t m,
                                             const double* __restrict__ gout, double* __restrict__ gdens,
                                             double* __restrict__ gsig)
{
    const int nc = t.n_ch;
    double g[kBwMaxCh] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int r = 0; r < nc && r < kBwMaxCh; ++r) g[r] = __ldg(gout + l * nc + r);
    const int64_t eb = search_key(E);
    const int32_t hb = t.H > 0 ? hash_bin(t, E, eb) : 0;
    const int32_t i0 = __ldg(t.moff + m), i1 = __ldg(t.moff + m + 1);
    for (int32_t i = i0; i < i1; ++i) {
        const int32_t s = __ldg(t.msp + i);
        const double N = __ldg(t.mden + i);
        const int64_t k = species_index(t, s, eb, hb);
        const int64_t p = __ldg(t.goff + s) + k;
        const double f = fraction_exact(E, __ldg(t.E + p), __ldg(t.E + p + 1));
        double dn = 0.0;
#pragma unroll
        for (int r = 0; r < kBwMaxCh; ++r) {
            if (r < nc) {
                const double s0 = sig_at<T>(t.sigma, p * nc + r);
                const double s1 = sig_at<T>(t.sigma, (p + 1) * nc + r);
                dn = dn + g[r] * interp_exact(s0, s1, f);
                atomicAdd(gsig + p * nc + r, N * (1.0 - f) * g[r]);
                atomicAdd(gsig + (p + 1) * nc + r, N * f * g[r]);
            }
        }
        atomicAdd(gdens + i, dn);
    }
}

// A total order of doubles (by value; -0 below +0) as signed 64-bit keys:
// positive values keep their bit pattern, negative ones flip the magnitude.
__device__ __forceinline__ int64_t order_key(double x)
{
    const int64_t b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}

__device__ __forceinline__ double from_order_key(int64_t k)
{
    return __longlong_as_double(k ^ ((k >> 63) & 0x7FFFFFFFFFFFFFFFLL));
}

// Per-warp staging of a sorted round of 32 lookups: energies, their order
// keys, cotangents, and the prefix sums over the sorted lanes of g_r and of
// (E - E_ref) g_r (entry c holds the sum over lanes [0, c)).
struct WarpStage {
    double E[32];
    int64_t key[32];
    double g[32][kBwMaxCh];
    double PG[33][kBwMaxCh];
    double PS[33][kBwMaxCh];
};

// First lane c in [lo, 32) whose key is >= k (32 if none); keys ascend.
__device__ __forceinline__ int lower_lane(const int64_t* key, int lo, int64_t k)
{
    int hi = 32;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (key[mid] < k) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <typename T>
__global__ void __launch_bounds__(kBwThreads) k_xs_backward_binned(Tables t, int64_t n,
                                                                   const double* __restrict__ Ein,
                                                                   const int32_t* __restrict__ mat,
                                                                   const int32_t* __restrict__ perm,
                                                                   const double* __restrict__ gout,
                                                                   double* __restrict__ gdens,
                                                                   double* __restrict__ gsig,
                                                                   unsigned long long* __restrict__ work,
                                                                   int32_t dens_in_smem)
{
    extern __shared__ double s_dens[];   // [nnz] when dens_in_smem
    __shared__ WarpStage stage[kBwWarps];
    const int nc = t.n_ch;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int32_t nnz = __ldg(t.moff + t.n_materials);
    if (dens_in_smem)
        for (int i = threadIdx.x; i < nnz; i += blockDim.x) s_dens[i] = 0.0;
    __syncthreads();
    WarpStage& ws = stage[wid];
    for (;;) {
        unsigned long long cb = 0ull;
        if (lane == 0) cb = atomicAdd(work, (unsigned long long)kBwChunk);
        cb = __shfl_sync(FULL, cb, 0);
        if ((int64_t)cb >= n) break;
#pragma unroll 1
        for (int rr = 0; rr < kBwChunk / 32; ++rr) {
            const int64_t j = (int64_t)cb + rr * 32 + lane;
            bool in = j < n;
            int64_t l = 0;
            double E = 0.0;
            int32_t m = -1;
            if (in) {
                l = __ldg(perm + j);
                if (MCX_IN_BOUNDS(l >= 0 && l < n, BC_PERM, l)) {
                    E = __ldg(Ein + l);
                    m = __ldg(mat + l);
                } else {
                    in = false;
                }
            }
            // valid: material in range and E finite (not NaN or infinite)
            const bool ok = in && m >= 0 && m < t.n_materials &&
                            (__double_as_longlong(E) & 0x7FF0000000000000LL) != 0x7FF0000000000000LL;
            const int32_t m0 = __shfl_sync(FULL, m, 0);
            if (!__all_sync(FULL, ok && m == m0)) {
                // mixed materials, an invalid lookup or the ragged tail
                if (in && m >= 0 && m < t.n_materials && E == E) backward_one<T>(t, l, E, m, gout, gdens, gsig);
                continue;
            }
            // ---- sort the 32 lookups by energy (ties by lookup index)
            int64_t key = order_key(E);
            int32_t pl = (int32_t)l;
#pragma unroll
            for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
                for (int jj = k >> 1; jj > 0; jj >>= 1) {
                    const int64_t ok2 = __shfl_xor_sync(FULL, key, jj);
                    const int32_t op = __shfl_xor_sync(FULL, pl, jj);
                    const bool up = (lane & k) == 0;
                    const bool lower = (lane & jj) == 0;
                    const bool other_smaller = ok2 < key || (ok2 == key && op < pl);
                    if ((lower == up) ? other_smaller : !other_smaller) {
                        key = ok2;
                        pl = op;
                    }
                }
            }
            const double Es = from_order_key(key);
            double g[kBwMaxCh];
#pragma unroll
            for (int r = 0; r < kBwMaxCh; ++r) g[r] = r < nc ? __ldg(gout + (int64_t)pl * nc + r) : 0.0;
            // ---- inclusive scans over the sorted lanes of g_r and (E - E_ref) g_r
            const double E_ref = __shfl_sync(FULL, Es, 0);
            const double E_top = __shfl_sync(FULL, Es, 31);
            const double d = Es - E_ref;
            double G[kBwMaxCh], S[kBwMaxCh];
#pragma unroll
            for (int r = 0; r < kBwMaxCh; ++r) {
                G[r] = g[r];
                S[r] = d * g[r];
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
                for (int r = 0; r < kBwMaxCh; ++r) {
                    if (r < nc) {
                        const double a = __shfl_up_sync(FULL, G[r], o), b = __shfl_up_sync(FULL, S[r], o);
                        if (lane >= o) {
                            G[r] = G[r] + a;
                            S[r] = S[r] + b;
                        }
                    }
                }
            }
            ws.E[lane] = Es;
            ws.key[lane] = key;
#pragma unroll
            for (int r = 0; r < kBwMaxCh; ++r) {
                ws.g[lane][r] = g[r];
                ws.PG[lane + 1][r] = G[r];
                ws.PS[lane + 1][r] = S[r];
                if (lane == 0) ws.PG[0][r] = ws.PS[0][r] = 0.0;
            }
            __syncwarp();
            const int64_t kb_lo = search_key(E_ref), kb_hi = search_key(E_top);
            const int32_t hb_lo = t.H > 0 ? hash_bin(t, E_ref, kb_lo) : 0;
            const int32_t hb_hi = t.H > 0 ? hash_bin(t, E_top, kb_hi) : 0;
            const int64_t key_lo = ws.key[0];
            const double span = E_top - E_ref;
            // ---- lanes over the material's species
            const int32_t i0 = __ldg(t.moff + m0), i1 = __ldg(t.moff + m0 + 1);
            for (int32_t ii = i0 + lane; ii < i1; ii += 32) {
                const int32_t s = __ldg(t.msp + ii);
                const double N = __ldg(t.mden + ii);
                const int64_t base = __ldg(t.goff + s);
                const int64_t last = __ldg(t.goff + s + 1) - base - 2;   // last interval
                const int64_t p_lo = species_index(t, s, kb_lo, hb_lo);
                const int64_t p_hi = species_index(t, s, kb_hi, hb_hi);
                const double* gE = t.E + base;
                double dn = 0.0;
                int a = 0;
                // lookups below the grid (only when p_lo == 0): f = 0 at point 0
                if (p_lo == 0 && key_lo < ebits(__ldg(gE))) {
                    a = lower_lane(ws.key, 0, ebits(__ldg(gE)));
#pragma unroll
                    for (int r = 0; r < kBwMaxCh; ++r) {
                        if (r < nc) {
                            const double A = ws.PG[a][r];
                            atomicAdd(gsig + base * nc + r, N * A);
                            dn = fma(A, sig_at<T>(t.sigma, base * nc + r), dn);
                        }
                    }
                }
                int64_t q = p_lo;
                while (a < 32) {
                    if (a > 0) q = bsearch_window(gE, q, p_hi, ws.key[a]);
                    const double g0 = __ldg(gE + q), g1 = __ldg(gE + q + 1);
                    const int64_t kg1 = ebits(g1);
                    // lanes [a, b) fall in interval q; at the last interval the
                    // lanes [c1, b) at or above the grid's top take f = 1
                    const int b = q < p_hi ? lower_lane(ws.key, a + 1, kg1) : 32;
                    const int c1 = (q == last && ws.key[b - 1] >= kg1) ? lower_lane(ws.key, a, kg1) : b;
                    const double w = __ldg(t.winv + base + q);
                    double A[kBwMaxCh], B[kBwMaxCh];
                    if (span <= 8.0 * (g1 - g0)) {
                        // f_l = (d_l + delta0) w over the run, from the prefix sums
                        const double d0 = E_ref - g0, d1 = g1 - E_ref;
#pragma unroll
                        for (int r = 0; r < kBwMaxCh; ++r) {
                            const double Gr = ws.PG[c1][r] - ws.PG[a][r];
                            const double Sr = ws.PS[c1][r] - ws.PS[a][r];
                            B[r] = w * fma(d0, Gr, Sr);
                            A[r] = w * fma(d1, Gr, -Sr);
                        }
                    } else {
                        // a warp spread over many intervals: lookup by lookup
#pragma unroll
                        for (int r = 0; r < kBwMaxCh; ++r) A[r] = B[r] = 0.0;
                        for (int c = a; c < c1; ++c) {
                            double f = (ws.E[c] - g0) * w;
                            const int64_t fb = __double_as_longlong(f);
                            if (fb < 0) f = 0.0;
                            if (fb > 0x3FF0000000000000LL) f = 1.0;
                            const double f1 = 1.0 - f;
#pragma unroll
                            for (int r = 0; r < kBwMaxCh; ++r) {
                                A[r] = fma(f1, ws.g[c][r], A[r]);
                                B[r] = fma(f, ws.g[c][r], B[r]);
                            }
                        }
                    }
                    if (c1 < b) {
#pragma unroll
                        for (int r = 0; r < kBwMaxCh; ++r) B[r] = B[r] + (ws.PG[b][r] - ws.PG[c1][r]);
                    }
                    const int64_t p = base + q;
#pragma unroll
                    for (int r = 0; r < kBwMaxCh; ++r) {
                        if (r < nc) {
                            const double s0 = sig_at<T>(t.sigma, p * nc + r);
                            const double s1 = sig_at<T>(t.sigma, (p + 1) * nc + r);
                            atomicAdd(gsig + p * nc + r, N * A[r]);
                            atomicAdd(gsig + (p + 1) * nc + r, N * B[r]);
                            dn = fma(A[r], s0, fma(B[r], s1, dn));
                        }
                    }
                    a = b;
                }
                if (dens_in_smem) atomicAdd(s_dens + ii, dn);
                else atomicAdd(gdens + ii, dn);
            }
            __syncwarp();   // the stage is rewritten by the next round
        }
    }
    if (dens_in_smem) {
        __syncthreads();
        for (int i = threadIdx.x; i < nnz; i += blockDim.x)
            if (s_dens[i] != 0.0) atomicAdd(gdens + i, s_dens[i]);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_xs_backward(Tables t, int64_t n, const double* __restrict__ Ein,
                                                     const int32_t* __restrict__ mat,
                                                     const double* __restrict__ gout,
                                                     double* __restrict__ gdens,
                                                     double* __restrict__ gsig)
{
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
         l += (int64_t)gridDim.x * blockDim.x) {
        const double E = __ldg(Ein + l);
        const int32_t m = __ldg(mat + l);
        if (m < 0 || m >= t.n_materials || E != E) continue;   // such lookups have no gradient
        backward_one<T>(t, l, E, m, gout, gdens, gsig);
    }
}

constexpr int kBwDensSmemMax = 6144;   // entries whose density sums fit in shared memory (48 KB)

}  // namespace

int launch_xs_backward(const Tables& t, int64_t n, const double* E, const int32_t* mat,
                       const double* grad_out, double* grad_dens, double* grad_sigma, int grid,
                       cudaStream_t st)
{
    if (t.precision == MCX_FP32)
        k_xs_backward<float><<<grid, 256, 0, st>>>(t, n, E, mat, grad_out, grad_dens, grad_sigma);
    else
        k_xs_backward<double><<<grid, 256, 0, st>>>(t, n, E, mat, grad_out, grad_dens, grad_sigma);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_xs_backward_binned(const Tables& t, int64_t nnz, int64_t n, const double* E, const int32_t* mat,
                              const int32_t* perm, const double* grad_out, double* grad_dens,
                              double* grad_sigma, int sm_count, unsigned long long* work, cudaStream_t st)
{
    if (!perm || !work || t.n_ch > kBwMaxCh) return -1;
    const int dens_smem = nnz <= kBwDensSmemMax ? 1 : 0;
    const size_t smem = dens_smem ? sizeof(double) * (size_t)nnz : 0;
    if (cudaMemsetAsync(work, 0, sizeof(unsigned long long), st) != cudaSuccess) return -1;
    auto kf = t.precision == MCX_FP32 ? k_xs_backward_binned<float> : k_xs_backward_binned<double>;
    if (cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -1;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kf, kBwThreads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    kf<<<sm_count * per_sm, kBwThreads, smem, st>>>(t, n, E, mat, perm, grad_out, grad_dens, grad_sigma, work,
                                                     dens_smem);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

MCX_BOUNDS_READER(bounds_error_adjoint)

}  // namespace mcx
