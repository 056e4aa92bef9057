// Stage kernels: scheme kWENO7, precision kMIXED.
#include "stage_launch.cuh"

namespace cosenu {
COSENU_INSTANTIATE_STAGE(kWENO7, kMIXED)
}  // namespace cosenu
