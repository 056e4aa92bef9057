// Stage kernels: scheme kWENO7, precision kFP64.
#include "stage_launch.cuh"

namespace cosenu {
COSENU_INSTANTIATE_STAGE(kWENO7, kFP64)
}  // namespace cosenu
