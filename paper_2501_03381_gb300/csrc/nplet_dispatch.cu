// Dispatch of the FP32 path by order: register-resident template instances
// for k <= 20, the generic kernel above.
#include "internal.cuh"

namespace thoi {

template <int K>
cudaError_t launch_reg_k(const NpletArgs& a, const Shape& sh, int num_sms, cudaStream_t s,
                         int* grid_out, int max_blocks);
cudaError_t launch_nplet_f32_gen(const NpletArgs& a, int num_sms, cudaStream_t s, int* grid_out,
                                 int max_blocks);

cudaError_t launch_nplet_f32(const NpletArgs& a, const Shape& sh, int num_sms, cudaStream_t s,
                             int* grid_out, int max_blocks) {
  switch (a.k) {
#define CASE_K(KK) \
  case KK: return launch_reg_k<KK>(a, sh, num_sms, s, grid_out, max_blocks);
    CASE_K(1) CASE_K(2) CASE_K(3) CASE_K(4) CASE_K(5) CASE_K(6) CASE_K(7) CASE_K(8) CASE_K(9)
    CASE_K(10) CASE_K(11) CASE_K(12) CASE_K(13) CASE_K(14) CASE_K(15) CASE_K(16) CASE_K(17)
    CASE_K(18) CASE_K(19) CASE_K(20)
#undef CASE_K
    default: return launch_nplet_f32_gen(a, num_sms, s, grid_out, max_blocks);
  }
}

}  // namespace thoi
