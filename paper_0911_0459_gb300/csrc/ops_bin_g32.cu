// Kernel instantiations for the binary model with the f populations and phi kept (g eliminated) (compiled separately).
#include "lb_ops_impl.cuh"

namespace lbk {
cudaError_t ops_bin_g32(OpKind op, const OpArgs& a, cudaStream_t s) { return ops_impl<MODEL_BINARY, SG32>(op, a, s); }
}  // namespace lbk
