// Instantiation of the FEWHA kernels for one precision.
#include "kernels.cuh"

namespace fewha {
ImplBase *make_impl_f32(const Plan &p) { return new Impl<float, float>(p); }
}  // namespace fewha
