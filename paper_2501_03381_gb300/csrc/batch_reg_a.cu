// Instantiations of the batched register-resident FP32 nplet kernel for orders 1..10.
#include "batch_reg.cuh"

namespace thoi {
THOI_BATCH_INSTANCE(1)
THOI_BATCH_INSTANCE(2)
THOI_BATCH_INSTANCE(3)
THOI_BATCH_INSTANCE(4)
THOI_BATCH_INSTANCE(5)
THOI_BATCH_INSTANCE(6)
THOI_BATCH_INSTANCE(7)
THOI_BATCH_INSTANCE(8)
THOI_BATCH_INSTANCE(9)
THOI_BATCH_INSTANCE(10)
}  // namespace thoi
