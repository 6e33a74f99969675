// Instantiations of the lane-group FP32 nplet kernel with 2 lanes for orders 13..16
// (an alternative to the one-thread kernel that the autotuner may pick).
#include "nplet_grp.cuh"

namespace thoi {
template cudaError_t launch_grp_k<13, 2>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_grp_k<14, 2>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_grp_k<15, 2>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_grp_k<16, 2>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
}  // namespace thoi
