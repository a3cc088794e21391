// fewha_read_probe: a streaming read of a device buffer by every SM, the
// measured denominator of the L2 roofline (the paper has no counterpart).
#include <cuda_runtime.h>

#include "../../include/fewha.h"

namespace {

// Grid-stride float4 reads; each CTA adds its threads' sums into one value
// so that no load can be dropped.
__global__ void __launch_bounds__(512) k_read_probe(const float4 *__restrict__ buf, long nvec, int passes,
                                                    float *__restrict__ sink)
{
    float acc = 0.f;
    const long stride = (long)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; p++) {
#pragma unroll 8
        for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nvec; i += stride) {
            const float4 v = __ldcg(buf + i);
            acc += (v.x + v.y) + (v.z + v.w);
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float part[16];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += part[w];
        sink[blockIdx.x] = s;
    }
}

}  // namespace

extern "C" int fewha_read_probe(const void *buf, long bytes, int reps, float *sink, cudaStream_t stream)
{
    if (!buf || !sink || bytes < 16 || (bytes & 15) || ((size_t)buf & 15) || reps < 1) return FEWHA_ERR_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FEWHA_ERR_CUDA;
    const int grid = 4 * nsm;  // four CTAs of 512 threads per SM
    k_read_probe<<<grid, 512, 0, stream>>>(static_cast<const float4 *>(buf), bytes / 16, reps, sink);
    return cudaGetLastError() == cudaSuccess ? FEWHA_OK : FEWHA_ERR_CUDA;
}
