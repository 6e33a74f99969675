// Instantiations of the register-resident FP32 nplet kernel for orders 17..18.
#include "nplet_reg.cuh"

namespace thoi {
template cudaError_t launch_reg_k<17>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_reg_k<18>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
}  // namespace thoi
