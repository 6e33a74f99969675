// Instantiations of the register-resident FP32 nplet kernel for orders 21..22 (the
// compiler spills a few registers here; the autotuner weighs them against the
// lane-group kernels).
#include "nplet_reg.cuh"

namespace thoi {
template cudaError_t launch_reg_k<21>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
template cudaError_t launch_reg_k<22>(const NpletArgs&, const Shape&, int, cudaStream_t, int*, int);
}  // namespace thoi
