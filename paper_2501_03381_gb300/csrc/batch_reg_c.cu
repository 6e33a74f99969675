// Instantiations of the batched register-resident FP32 nplet kernel for orders 16..20.
#include "batch_reg.cuh"

namespace thoi {
THOI_BATCH_INSTANCE(16)
THOI_BATCH_INSTANCE(17)
THOI_BATCH_INSTANCE(18)
THOI_BATCH_INSTANCE(19)
THOI_BATCH_INSTANCE(20)
}  // namespace thoi
