// Operator kernels instantiated for dim = 2, float arithmetic.
#include "ops_impl.cuh"

namespace dg {
DG_INSTANTIATE_OPS(2, float)
}  // namespace dg
