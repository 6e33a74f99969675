// Dispatch of the FP32 path by order: one-thread register kernels for
// k <= 20, lane-group register kernels for 21 <= k <= 32 (2 lanes per nplet
// up to 24, 4 lanes above), the generic kernel beyond.
#include "internal.cuh"

namespace thoi {

template <int K>
cudaError_t launch_reg_k(const NpletArgs& a, const Shape& sh, int num_sms, cudaStream_t s,
                         int* grid_out, int max_blocks);
template <int K, int G>
cudaError_t launch_grp_k(const NpletArgs& a, const Shape& sh, int num_sms, cudaStream_t s,
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
#define CASE_G(KK, GG) \
  case KK: return launch_grp_k<KK, GG>(a, sh, num_sms, s, grid_out, max_blocks);
    CASE_G(21, 2) CASE_G(22, 2) CASE_G(23, 2) CASE_G(24, 2) CASE_G(25, 4) CASE_G(26, 4)
    CASE_G(27, 4) CASE_G(28, 4) CASE_G(29, 4) CASE_G(30, 4) CASE_G(31, 4) CASE_G(32, 4)
#undef CASE_G
    default: return launch_nplet_f32_gen(a, num_sms, s, grid_out, max_blocks);
  }
}

}  // namespace thoi
