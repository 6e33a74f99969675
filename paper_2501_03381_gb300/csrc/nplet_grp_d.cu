// Instantiations of the lane-group FP32 nplet kernel for orders 29..32.
#include "nplet_grp.cuh"

namespace thoi {
template cudaError_t launch_grp_k<29, 4>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_grp_k<30, 4>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_grp_k<31, 4>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_grp_k<32, 4>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
}  // namespace thoi
