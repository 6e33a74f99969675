// Instantiations of the two-level prefix-shared FP32 nplet kernel for orders 17..20.
#include "nplet_pfx2.cuh"

namespace thoi {
template cudaError_t launch_pfx2_k<17>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx2_k<18>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx2_k<19>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx2_k<20>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
}  // namespace thoi
