// Operator kernels instantiated for dim = 2, double arithmetic.
#include "ops_impl.cuh"

namespace dg {
DG_INSTANTIATE_OPS(2, double)
}  // namespace dg
