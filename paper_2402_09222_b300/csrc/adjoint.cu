// adjoint.cu -- backward pass of the macroscopic lookup (compiled with
// --fmad=false).  The lookup is linear in the densities N_j and in the table
// entries s[k], s[k+1]:  Sigma_r = sum_j N_j ((1 - f) s_r[k] + f s_r[k+1]),
// so for a cotangent g_r of the output
//   dL/dN_j       = sum_r g_r sigma_{r,j}(E)
//   dL/ds_r[k]   += N_j (1 - f) g_r,     dL/ds_r[k+1] += N_j f g_r.
// Each lookup adds its contributions with FP64 atomics.
#include "kernels.h"
#include "xs_exact.cuh"

namespace mcx {

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_xs_backward(Tables t, int64_t n, const double* __restrict__ Ein,
                                                     const int32_t* __restrict__ mat,
                                                     const double* __restrict__ gout,
                                                     double* __restrict__ gdens,
                                                     double* __restrict__ gsig)
{
    const int nc = t.n_ch;
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
         l += (int64_t)gridDim.x * blockDim.x) {
        const double E = __ldg(Ein + l);
        const int32_t m = __ldg(mat + l);
        if (m < 0 || m >= t.n_materials || E != E) continue;   // such lookups have no gradient
        double g[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int r = 0; r < nc && r < 5; ++r) g[r] = __ldg(gout + l * nc + r);
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
            for (int r = 0; r < 5; ++r) {
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
}

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

}  // namespace mcx
