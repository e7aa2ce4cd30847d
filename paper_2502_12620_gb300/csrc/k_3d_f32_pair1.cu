// The cell-pair FP32 stage kernel for 3D blocks of 8^3 cells at p = 1.
#include "stage_pair.cuh"

namespace dgf {
template cudaError_t stage_pair_launch<1>(const StageArgs<3, 1, float>&, int, bool, bool, cudaStream_t, int);
template int stage_pair_blocks_per_sm<1>(int);
template cudaError_t stage_pair_launch_batch<1>(const StageArgs<3, 1, float>&, int, bool, cudaStream_t);
}  // namespace dgf
