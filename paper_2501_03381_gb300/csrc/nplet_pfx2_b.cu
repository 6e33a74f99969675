// Instantiations of the two-level prefix-shared FP32 nplet kernel for orders 13..16.
#include "nplet_pfx2.cuh"

namespace thoi {
template cudaError_t launch_pfx2_k<13>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx2_k<14>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx2_k<15>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_pfx2_k<16>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
}  // namespace thoi
