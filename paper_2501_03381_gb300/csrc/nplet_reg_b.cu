// Instantiations of the register-resident FP32 nplet kernel for orders 11..14.
#include "nplet_reg.cuh"

namespace thoi {
template cudaError_t launch_reg_k<11>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_reg_k<12>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_reg_k<13>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_reg_k<14>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
}  // namespace thoi
