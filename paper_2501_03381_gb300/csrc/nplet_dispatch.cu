// Dispatch of the FP32 path by order: one-thread register kernels for
// k <= 24, lane-group register kernels for 13 <= k <= 32 (2 lanes per nplet
// up to 24, 4 lanes from 21), the generic kernel beyond.  Without a tuned
// shape, orders up to 20 use one thread per nplet, 21..24 two lanes, 25..32
// four lanes.
#include "internal.cuh"

namespace thoi {

template <int K>
cudaError_t launch_reg_k(const NpletArgs& a, const Shape& sh, int num_sms, cudaStream_t s,
                         int* grid_out, int max_blocks);
template <int K>
cudaError_t launch_pfx_k(const NpletArgs& a, const Shape& sh, int num_sms, cudaStream_t s,
                         int* grid_out, int max_blocks);
template <int K>
cudaError_t launch_pfx2_k(const NpletArgs& a, const Shape& sh, int num_sms, cudaStream_t s,
                          int* grid_out, int max_blocks);
template <int K, int G>
cudaError_t launch_grp_k(const NpletArgs& a, const Shape& sh, int num_sms, cudaStream_t s,
                         int* grid_out, int max_blocks);
cudaError_t launch_nplet_f32_gen(const NpletArgs& a, int num_sms, cudaStream_t s, int* grid_out,
                                 int max_blocks);

Shape default_shape(int k) {
  Shape s;
  s.blocks_per_sm = 0;
  s.chunk = 8;
  s.lanes = k <= 24 ? 1 : (k <= 32 ? 4 : 1);
  s.prefix = 0;
  return s;
}

bool shape_available(int k, int lanes) {
  if (lanes == 1) return true;  // one-thread kernel for k <= 20, generic above
  if (lanes == 2) return k >= 13 && k <= 24;
  if (lanes == 4) return k >= 21 && k <= 32;
  return false;
}

static unsigned long long binom_u(int n, int k) {
  if (k < 0 || k > n) return 0;
  unsigned __int128 r = 1;
  for (int i = 1; i <= k; i++) r = r * (unsigned)(n - k + i) / (unsigned)i;
  return (unsigned long long)r;
}

cudaError_t launch_nplet_f32(const NpletArgs& a, const Shape& sh, int num_sms, cudaStream_t s,
                             int* grid_out, int max_blocks) {
  // the prefix-shared kernel covers whole orders only
  if (sh.prefix && a.k >= KPFX_MIN && a.k <= (sh.prefix >= 2 ? KPFX2_MAX : KPFX_MAX) &&
      a.rank_begin == 0 && a.rank_end == binom_u(a.N, a.k)) {
    switch (a.k) {
#define CASE_P(KK)                                                                  \
  case KK:                                                                          \
    return sh.prefix >= 2 ? launch_pfx2_k<KK>(a, sh, num_sms, s, grid_out, max_blocks) \
                          : launch_pfx_k<KK>(a, sh, num_sms, s, grid_out, max_blocks);
      CASE_P(3) CASE_P(4) CASE_P(5) CASE_P(6) CASE_P(7) CASE_P(8) CASE_P(9) CASE_P(10)
      CASE_P(11) CASE_P(12) CASE_P(13) CASE_P(14) CASE_P(15) CASE_P(16) CASE_P(17) CASE_P(18)
      CASE_P(19) CASE_P(20)
#undef CASE_P
      case 21: return launch_pfx2_k<21>(a, sh, num_sms, s, grid_out, max_blocks);
      case 22: return launch_pfx2_k<22>(a, sh, num_sms, s, grid_out, max_blocks);
      case 23: return launch_pfx2_k<23>(a, sh, num_sms, s, grid_out, max_blocks);
      case 24: return launch_pfx2_k<24>(a, sh, num_sms, s, grid_out, max_blocks);
      default: break;
    }
  }
  // a prefix shape's chunk counts prefixes per fetch: where the dense kernels
  // run instead (a sub-range, an order the prefix kernels do not cover) they
  // take their own default shape
  if (sh.prefix) return launch_nplet_f32(a, default_shape(a.k), num_sms, s, grid_out, max_blocks);
  const int lanes = shape_available(a.k, sh.lanes) ? sh.lanes : default_shape(a.k).lanes;
  if (lanes == 2) {
    switch (a.k) {
#define CASE_G(KK) \
  case KK: return launch_grp_k<KK, 2>(a, sh, num_sms, s, grid_out, max_blocks);
      CASE_G(13) CASE_G(14) CASE_G(15) CASE_G(16) CASE_G(17) CASE_G(18) CASE_G(19) CASE_G(20)
      CASE_G(21) CASE_G(22) CASE_G(23) CASE_G(24)
#undef CASE_G
      default: break;
    }
  }
  if (lanes == 4) {
    switch (a.k) {
#define CASE_G(KK) \
  case KK: return launch_grp_k<KK, 4>(a, sh, num_sms, s, grid_out, max_blocks);
      CASE_G(21) CASE_G(22) CASE_G(23) CASE_G(24)
      CASE_G(25) CASE_G(26) CASE_G(27) CASE_G(28) CASE_G(29) CASE_G(30) CASE_G(31) CASE_G(32)
#undef CASE_G
      default: break;
    }
  }
  switch (a.k) {
#define CASE_K(KK) \
  case KK: return launch_reg_k<KK>(a, sh, num_sms, s, grid_out, max_blocks);
    CASE_K(1) CASE_K(2) CASE_K(3) CASE_K(4) CASE_K(5) CASE_K(6) CASE_K(7) CASE_K(8) CASE_K(9)
    CASE_K(10) CASE_K(11) CASE_K(12) CASE_K(13) CASE_K(14) CASE_K(15) CASE_K(16) CASE_K(17)
    CASE_K(18) CASE_K(19) CASE_K(20) CASE_K(21) CASE_K(22) CASE_K(23) CASE_K(24)
#undef CASE_K
    default: return launch_nplet_f32_gen(a, num_sms, s, grid_out, max_blocks);
  }
}

}  // namespace thoi
