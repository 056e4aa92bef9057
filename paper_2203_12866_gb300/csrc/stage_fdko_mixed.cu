// Stage kernels: scheme kFDKO, precision kMIXED.
#include "stage_launch.cuh"

namespace cosenu {
COSENU_INSTANTIATE_STAGE(kFDKO, kMIXED)
}  // namespace cosenu
