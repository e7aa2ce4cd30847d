// Kernel instantiations for dimension 2, element type float.
#include "kernels_inst.cuh"

namespace dgf {
DGF_INSTANTIATE(2, float)
}  // namespace dgf
