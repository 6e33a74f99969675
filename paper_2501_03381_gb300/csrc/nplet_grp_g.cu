// Instantiations of the lane-group FP32 nplet kernel with 4 lanes for orders
// 21..24 (an alternative to 2 lanes that the autotuner may pick).
#include "nplet_grp.cuh"

namespace thoi {
template cudaError_t launch_grp_k<21, 4>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_grp_k<22, 4>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_grp_k<23, 4>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_grp_k<24, 4>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
}  // namespace thoi
