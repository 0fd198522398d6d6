// Fused step kernels of every tile shape, FP64 and double-single storage.
#include "step_shapes.inl"

namespace lbmfvm_fv {
LBMFVM_STEP_INSTANTIATE(double)
LBMFVM_STEP_INSTANTIATE(lbmfvm_dev::dsf)
}  // namespace lbmfvm_fv
