// Instantiations of the batched register-resident FP32 nplet kernel for orders 11..15.
#include "batch_reg.cuh"

namespace thoi {
THOI_BATCH_INSTANCE(11)
THOI_BATCH_INSTANCE(12)
THOI_BATCH_INSTANCE(13)
THOI_BATCH_INSTANCE(14)
THOI_BATCH_INSTANCE(15)
}  // namespace thoi
