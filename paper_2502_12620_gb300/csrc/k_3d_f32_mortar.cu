// Mortar-mode stage kernels (reading R15) for dimension 3, element type float.
#include "kernels_inst.cuh"

namespace dgf {
DGF_INSTANTIATE_MORTAR(3, float)
}  // namespace dgf
