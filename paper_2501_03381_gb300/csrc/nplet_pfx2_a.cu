// Instantiations of the two-level prefix-shared FP32 nplet kernel for orders 3..12.
#include "nplet_pfx2.cuh"

namespace thoi {
template cudaError_t launch_pfx2_k<3>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx2_k<4>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx2_k<5>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx2_k<6>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx2_k<7>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx2_k<8>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx2_k<9>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx2_k<10>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx2_k<11>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx2_k<12>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
}  // namespace thoi
