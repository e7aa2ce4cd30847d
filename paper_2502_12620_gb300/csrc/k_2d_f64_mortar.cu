// Mortar-mode stage kernels (reading R15) for dimension 2, element type double.
#include "kernels_inst.cuh"

namespace dgf {
DGF_INSTANTIATE_MORTAR(2, double)
}  // namespace dgf
