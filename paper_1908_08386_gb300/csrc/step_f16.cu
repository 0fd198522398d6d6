// Fused step kernels of every tile shape, FP16 and BF16 storage.
#include "step_shapes.inl"

namespace lbmfvm_fv {
LBMFVM_STEP_INSTANTIATE(__half)
LBMFVM_STEP_INSTANTIATE(__nv_bfloat16)
}  // namespace lbmfvm_fv
