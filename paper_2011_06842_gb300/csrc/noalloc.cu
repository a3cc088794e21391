// fewha_apply_op_noalloc: the operator application y = M x with its scratch
// in a statically reserved device array instead of handle-owned allocations.
// Who needs it and the sharing rules are stated with its declaration in
// include/fewha.h.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace {

// One array per device.  It lives in this translation unit's module, which
// CUDA's lazy module loading brings onto a device the first time a symbol of
// it is looked up there: fewha_create does that (noalloc_prepare), so the
// array is reserved while creating a handle is still allowed to allocate.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FEWHA_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch on the current device.  Looked up on
// every call rather than cached: a cached pointer would outlive a device
// reset or a new primary context.  Once the module is loaded the lookup
// allocates nothing.  (The host-side name of the array is only a stand-in,
// never a device address.)
int scratch_address(void **out)
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FEWHA_ERR_CUDA;
    *out = p;
    return FEWHA_OK;
}

bool aligned16(const void *p) { return ((size_t)p & 15) == 0; }

}  // namespace

namespace fewha {

int noalloc_prepare()
{
    void *p = nullptr;
    return scratch_address(&p);
}

}  // namespace fewha

extern "C" int fewha_apply_op_noalloc(void *handle, const void *x, void *y, cudaStream_t stream)
{
    if (!handle || !x || !y || x == y || !aligned16(x) || !aligned16(y)) return FEWHA_ERR_ARG;
    // the scratch used is the current device's: it must be the device whose
    // tables the handle holds
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FEWHA_ERR_CUDA;
    if (dev != fewha::handle_device(handle)) return FEWHA_ERR_ARG;
    void *scratch = nullptr;
    const int st = scratch_address(&scratch);
    if (st != FEWHA_OK) return st;
    return fewha::handle_impl(handle)->apply_in_scratch(x, y, scratch, FEWHA_NOALLOC_SCRATCH_BYTES, stream);
}
