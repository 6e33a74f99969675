// Instantiations of the register-resident FP32 nplet kernel for orders 15..16.
#include "nplet_reg.cuh"

namespace thoi {
template cudaError_t launch_reg_k<15>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_reg_k<16>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
}  // namespace thoi
