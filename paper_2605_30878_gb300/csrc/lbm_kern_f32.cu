// FP32 instantiation of every kernel launcher.
#include "lbm_launch.cuh"

namespace lbmgpu {
template struct Launch<float>;
}  // namespace lbmgpu
