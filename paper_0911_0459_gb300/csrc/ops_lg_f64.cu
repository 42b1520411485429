// Kernel instantiations for one model x storage pair (compiled separately).
#include "lb_ops_impl.cuh"

namespace lbk {
cudaError_t ops_lg_f64(OpKind op, const OpArgs& a, cudaStream_t s) { return ops_impl<MODEL_LG, SF64>(op, a, s); }
}  // namespace lbk
