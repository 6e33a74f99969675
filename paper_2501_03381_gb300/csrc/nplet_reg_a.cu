// Instantiations of the register-resident FP32 nplet kernel for orders 1..10.
#include "nplet_reg.cuh"

namespace thoi {
template cudaError_t launch_reg_k<1>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_reg_k<2>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_reg_k<3>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_reg_k<4>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_reg_k<5>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_reg_k<6>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_reg_k<7>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_reg_k<8>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_reg_k<9>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_reg_k<10>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
}  // namespace thoi
