// Instantiation of the two-, three- and four-level prefix-shared FP32 nplet
// kernels for order 24 (beyond the one-level kernel's orders).
#include "nplet_pfx2.cuh"

namespace thoi {
template cudaError_t launch_pfx2_k<24>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
}  // namespace thoi
