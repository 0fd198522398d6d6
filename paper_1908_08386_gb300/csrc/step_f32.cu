// Fused step kernels of every tile shape, FP32 storage.
#include "step_shapes.inl"

namespace lbmfvm_fv {
LBMFVM_STEP_INSTANTIATE(float)
}  // namespace lbmfvm_fv
