// Kernel instantiations for dimension 3, element type float.
#include "kernels_inst.cuh"

namespace dgf {
DGF_INSTANTIATE(3, float)
}  // namespace dgf
