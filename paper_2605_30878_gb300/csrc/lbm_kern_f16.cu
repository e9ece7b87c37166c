// FP32 arithmetic with FP16 population storage: instantiation of every kernel launcher.
#include "lbm_launch_impl.cuh"

namespace lbmgpu {
template struct Launch<float, __half>;
}  // namespace lbmgpu
