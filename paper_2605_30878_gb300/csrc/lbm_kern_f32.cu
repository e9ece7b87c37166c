// FP32 arithmetic and storage: instantiation of every kernel launcher.
#include "lbm_launch_impl.cuh"

namespace lbmgpu {
template struct Launch<float, float>;
}  // namespace lbmgpu
