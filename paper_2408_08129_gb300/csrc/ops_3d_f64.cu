// Operator kernels instantiated for dim = 3, double arithmetic.
#include "ops_impl.cuh"

namespace dg {
DG_INSTANTIATE_OPS(3, double)
}  // namespace dg
