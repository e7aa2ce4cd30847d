// Mortar-mode stage kernels (reading R15) for dimension 2, element type float.
#include "kernels_inst.cuh"

namespace dgf {
DGF_INSTANTIATE_MORTAR(2, float)
}  // namespace dgf
