// Kernel instantiations for the binary model with the state kept as six FP32
// moments per node (compiled separately).
#include "lb_ops_impl.cuh"

namespace lbk {
cudaError_t ops_bin_m32(OpKind op, const OpArgs& a, cudaStream_t s) { return ops_impl<MODEL_BINARY, SM32>(op, a, s); }
}  // namespace lbk
