// Instantiation of the FEWHA kernels for one precision.
#include "kernels.cuh"

namespace fewha {
ImplBase *make_impl_bf16(const Plan &p) { return new Impl<float, __nv_bfloat16>(p); }
}  // namespace fewha
