// Kernel instantiations for dimension 2, element type double.
#include "kernels_inst.cuh"

namespace dgf {
DGF_INSTANTIATE(2, double)
}  // namespace dgf
