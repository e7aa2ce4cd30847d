// Kernel instantiations for dimension 3, element type double.
#include "kernels_inst.cuh"

namespace dgf {
DGF_INSTANTIATE(3, double)
}  // namespace dgf
