// Kernel instantiations for the binary model with FP16 deviations in blocks of
// 32 nodes (compiled separately).
#include "lb_ops_impl.cuh"

namespace lbk {
cudaError_t ops_bin_f16b(OpKind op, const OpArgs& a, cudaStream_t s) { return ops_impl<MODEL_BINARY, SF16B>(op, a, s); }
}  // namespace lbk
