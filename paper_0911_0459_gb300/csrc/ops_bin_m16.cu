// Kernel instantiations for the binary model with the state kept as FP16 moments with an FP32 phi (compiled separately).
#include "lb_ops_impl.cuh"

namespace lbk {
cudaError_t ops_bin_m16(OpKind op, const OpArgs& a, cudaStream_t s) { return ops_impl<MODEL_BINARY, SM16>(op, a, s); }
}  // namespace lbk
