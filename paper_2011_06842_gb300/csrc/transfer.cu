// Host <-> device traffic of a time step without the copy engines.  On this
// part page-locked host memory is mapped into the device's address space and
// reached over the chip-to-chip link, so a kernel can read a frame's slopes
// from it (zero-copy) and write the solution back to it.  Each copy-engine
// transfer on the stream costs a hand-off between the engine and the SMs in
// both directions; reading and writing from the kernels avoids both (not part
// of the paper's method: how a time step's inputs and result cross the link).
#include <cuda_runtime.h>

#include "../../include/fewha.h"

namespace fewha {

// The address under which the device reaches p: p itself for device and
// managed memory, the mapped address for page-locked host memory
// (cudaHostAlloc, cudaMallocHost, cudaHostRegister); nullptr for pageable
// host memory and unknown pointers, which kernels must not touch.
const void *fewha_device_view(const void *p)
{
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // clear the error state of the failed query
        return nullptr;
    }
    switch (a.type) {
    case cudaMemoryTypeDevice:
    case cudaMemoryTypeManaged:
        return p;
    case cudaMemoryTypeHost:
        return a.devicePointer;
    default:
        return nullptr;
    }
}

}  // namespace fewha

namespace {

__global__ void __launch_bounds__(256) k_store(const float4 *__restrict__ src, float4 *__restrict__ dst, long n16)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n16; i += (long)gridDim.x * blockDim.x)
        dst[i] = __ldcg(src + i);
}

}  // namespace

extern "C" int fewha_store(void *dst, const void *src, long bytes, cudaStream_t stream)
{
    if (!dst || !src || bytes < 16 || (bytes & 15) || ((size_t)src & 15)) return FEWHA_ERR_ARG;
    void *d = const_cast<void *>(fewha::fewha_device_view(dst));
    const void *s = fewha::fewha_device_view(src);
    if (!d || !s || ((size_t)d & 15) || ((size_t)s & 15)) return FEWHA_ERR_ARG;
    const char *sb = static_cast<const char *>(s), *db = static_cast<const char *>(d);
    if (sb < db + bytes && db < sb + bytes) return FEWHA_ERR_ARG;  // no overlap
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FEWHA_ERR_CUDA;
    const long n16 = bytes / 16;
    long grid = (n16 + 255) / 256;
    if (grid > 2L * nsm) grid = 2L * nsm;
    k_store<<<(unsigned)grid, 256, 0, stream>>>(static_cast<const float4 *>(s), static_cast<float4 *>(d), n16);
    return cudaGetLastError() == cudaSuccess ? FEWHA_OK : FEWHA_ERR_CUDA;
}
