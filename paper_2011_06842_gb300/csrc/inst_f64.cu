// Instantiation of the FEWHA kernels for one precision.
#include "kernels.cuh"

namespace fewha {
ImplBase *make_impl_f64(const Plan &p) { return new Impl<double, double>(p); }
}  // namespace fewha
