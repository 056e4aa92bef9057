// Stage kernels: scheme kFDKO3, precision kFP64.
#include "stage_launch.cuh"

namespace cosenu {
COSENU_INSTANTIATE_STAGE(kFDKO3, kFP64)
}  // namespace cosenu
