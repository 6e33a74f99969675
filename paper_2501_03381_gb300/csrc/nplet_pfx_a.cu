// Instantiations of the prefix-shared FP32 nplet kernel for orders 3..12.
#include "nplet_pfx.cuh"

namespace thoi {
template cudaError_t launch_pfx_k<3>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx_k<4>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx_k<5>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx_k<6>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx_k<7>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx_k<8>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx_k<9>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx_k<10>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx_k<11>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx_k<12>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
}  // namespace thoi
