// FP64 instantiation of every kernel launcher.
#include "lbm_launch.cuh"

namespace lbmgpu {
template struct Launch<double>;
}  // namespace lbmgpu
