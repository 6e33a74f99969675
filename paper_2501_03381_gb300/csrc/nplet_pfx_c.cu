// Instantiations of the prefix-shared FP32 nplet kernel for orders 17..20.
#include "nplet_pfx.cuh"

namespace thoi {
template cudaError_t launch_pfx_k<17>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx_k<18>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx_k<19>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx_k<20>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
}  // namespace thoi
