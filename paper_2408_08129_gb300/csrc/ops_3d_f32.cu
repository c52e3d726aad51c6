// Operator kernels instantiated for dim = 3, float arithmetic.
#include "ops_impl.cuh"

namespace dg {
DG_INSTANTIATE_OPS(3, float)
}  // namespace dg
