// Stage kernels: scheme kFDKO, precision kFP64.
#include "stage_launch.cuh"

namespace cosenu {
COSENU_INSTANTIATE_STAGE(kFDKO, kFP64)
}  // namespace cosenu
