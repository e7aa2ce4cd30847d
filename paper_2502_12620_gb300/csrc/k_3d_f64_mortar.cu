// Mortar-mode stage kernels (reading R15) for dimension 3, element type double.
#include "kernels_inst.cuh"

namespace dgf {
DGF_INSTANTIATE_MORTAR(3, double)
}  // namespace dgf
