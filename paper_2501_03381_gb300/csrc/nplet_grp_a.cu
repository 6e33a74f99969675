// Instantiations of the lane-group FP32 nplet kernel for orders 21..22.
#include "nplet_grp.cuh"

namespace thoi {
template cudaError_t launch_grp_k<21, 2>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_grp_k<22, 2>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
}  // namespace thoi
