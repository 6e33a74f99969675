// Instantiations of the register-resident FP32 nplet kernel for orders 23..24 (the
// compiler spills a few registers here; the autotuner weighs them against the
// lane-group kernels).
#include "nplet_reg.cuh"

namespace thoi {
template cudaError_t launch_reg_k<23>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_reg_k<24>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
}  // namespace thoi
