// Instantiations of the lane-group FP32 nplet kernel for orders 25..28.
#include "nplet_grp.cuh"

namespace thoi {
template cudaError_t launch_grp_k<25, 4>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_grp_k<26, 4>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_grp_k<27, 4>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_grp_k<28, 4>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
}  // namespace thoi
