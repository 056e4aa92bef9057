// Stage kernels: scheme kFDKO3, precision kMIXED.
#include "stage_launch.cuh"

namespace cosenu {
COSENU_INSTANTIATE_STAGE(kFDKO3, kMIXED)
}  // namespace cosenu
