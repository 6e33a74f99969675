// Instantiations of the register-resident FP32 nplet kernel for orders 19..20.
#include "nplet_reg.cuh"

namespace thoi {
template cudaError_t launch_reg_k<19>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_reg_k<20>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
}  // namespace thoi
