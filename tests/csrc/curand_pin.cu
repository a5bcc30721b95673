// Test helper: runs cuRAND's Philox4x32-10 device function on given counters
// and keys, so the library's own Philox can be pinned against it.
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void k_curand_philox(const uint4* ctr, const uint2* key, uint4* out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

extern "C" int curand_philox_blocks(const void* ctr, const void* key, void* out, int n)
{
    if (n <= 0) return 0;
    k_curand_philox<<<(n + 127) / 128, 128>>>((const uint4*)ctr, (const uint2*)key, (uint4*)out, n);
    if (cudaGetLastError() != cudaSuccess) return -1;
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : -1;
}
