// fewha_apply_op_noalloc: the operator application y = M x with its scratch
// in a statically reserved device array instead of handle-owned allocations.
// See include/fewha.h for who needs it and the sharing rules.
#include <cuda_runtime.h>

#include <mutex>

#include "kernels.cuh"

namespace {

// One array per device, reserved when the library's module is loaded.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FEWHA_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once
// per device; the host-side name is only a stand-in, never a device pointer).
int scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FEWHA_ERR_CUDA;
    std::lock_guard<std::mutex> g(g_lock);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FEWHA_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return FEWHA_OK;
}

bool aligned16(const void *p) { return ((size_t)p & 15) == 0; }

}  // namespace

extern "C" int fewha_apply_op_noalloc(void *handle, const void *x, void *y, cudaStream_t stream)
{
    if (!handle || !x || !y || x == y || !aligned16(x) || !aligned16(y)) return FEWHA_ERR_ARG;
    void *scratch = nullptr;
    int st = scratch_address(&scratch);
    if (st != FEWHA_OK) return st;
    return fewha::handle_impl(handle)->apply_in_scratch(x, y, scratch, FEWHA_NOALLOC_SCRATCH_BYTES, stream);
}
