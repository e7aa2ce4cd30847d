// The cell-pair FP32 stage kernel for 3D blocks of 8^3 cells at p = 2.
#include "stage_pair.cuh"

namespace dgf {
template cudaError_t stage_pair_launch<2>(const StageArgs<3, 2, float>&, int, bool, bool, cudaStream_t, int);
template int stage_pair_blocks_per_sm<2>(int);
template cudaError_t stage_pair_launch_batch<2>(const StageArgs<3, 2, float>&, int, bool, cudaStream_t);
}  // namespace dgf
