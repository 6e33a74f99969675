// Instance of the persistent batched FP32 nplet kernel for orders 1..8.
#include "batch_fused.cuh"

namespace thoi {
template cudaError_t bfused_launch<1, 8>(bool, const BatchFArgs&, int, int, int, cudaStream_t, int*);
}  // namespace thoi
