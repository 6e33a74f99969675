// FP64 nplet kernel: the THOI_F64 path and the re-factor of the nplets the
// FP32 path flagged.  Matrices live in shared memory: for small orders one
// nplet per thread (each thread's k x k matrix interleaved across the block,
// entry e of thread t at mat[e * NT + t]); for large orders G lanes share one
// nplet's matrix (f64g_body), so that a block still holds enough warps to
// keep the FP64 pipe busy.  FP64 arithmetic runs at a small fraction of the
// FP32 rate on this GPU, so shared-memory bandwidth is ample; what matters is
// latency and the number of resident warps.
//
// Same quantities as the FP32 kernels: R_S = Lh D Lh^T, log det R_S =
// sum log D_p, the unit-lower inverse V column by column, and
// p_j = (R_S^-1)_jj = 1/D_j + sum_{i>j} V_ij^2 / D_i.  A pivot D_p <= 0 marks
// the nplet not positive definite.
#include "nplet_f64.cuh"

namespace thoi {

template <int NT, int G, bool LIST, typename M>
__global__ void __launch_bounds__(NT) k_nplet_f64s(const NpletArgs a, double* __restrict__ b64,
                                                   unsigned long long bstride) {
  extern __shared__ __align__(16) unsigned char smem[];
  if constexpr (G == 1) f64s_body<NT, LIST, M>(a, b64, bstride, smem);
  else f64g_body<NT, G, LIST, M>(a, b64, bstride, smem);
}

// Lanes per nplet and shared memory for (N, k): the fewest lanes per nplet
// (one thread per nplet first) whose block stays within F64_SMEM_TARGET, so
// that two blocks (eight warps) share an SM.  Fewer lanes per nplet leave
// fewer of them idle in the triangular loops, and the FP64 pipe charges a
// warp instruction whatever its active lanes; two blocks per SM keep it fed.
// (Measured on N = 30: orders 18, 20, 22, 25, 28 each fastest with the G
// this picks, against 72 KB, 100 KB and 128 KB targets.)
constexpr size_t F64_SMEM_TARGET = 112 * 1024;
constexpr int F64_NT = 128;

F64Cfg f64_config(int N, int k) {
  F64Cfg c;
  const SmemLayout L = smem_layout(N, k, row_stride(N), sizeof(double), 8, 0);
  const size_t s1 = L.total + (size_t)(k * (k + 1) / 2) * sizeof(double) * F64_NT;
  if (s1 <= F64_SMEM_TARGET) {
    c.G = 1;
    c.smem = s1;
    return c;
  }
  for (int G = 2; G <= 32; G <<= 1) {
    const size_t sg = f64g_smem(N, k, F64_NT, G);
    if (sg <= F64_SMEM_TARGET || G == 32) {
      c.G = G;
      c.smem = sg;
      return c;
    }
  }
  c.G = 32;
  c.smem = f64g_smem(N, k, F64_NT, 32);
  return c;
}

template <int G, bool LIST>
static cudaError_t launch_f64s_t(const NpletArgs& a, double* b64, unsigned long long bstride,
                                 size_t sm, int num_sms, cudaStream_t s, int* grid_out,
                                 int max_blocks) {
  constexpr int NT = F64_NT;
  void (*fn)(const NpletArgs, double*, unsigned long long);
  if (a.N > 32) fn = k_nplet_f64s<NT, G, LIST, unsigned long long>;
  else fn = k_nplet_f64s<NT, G, LIST, unsigned>;
  int occ = 0;
  cudaError_t e = occupancy_cached((const void*)fn, NT, sm, &occ);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  long long grid = (long long)num_sms * occ;
  if (!LIST) {
    const unsigned long long n = a.rank_end - a.rank_begin;
    const unsigned long long per_block = NT / G;
    const long long need = (long long)((n + per_block - 1) / per_block);
    if (need < grid) grid = need > 0 ? need : 1;
  }
  if (grid > max_blocks) grid = max_blocks;
  fn<<<(unsigned)grid, NT, sm, s>>>(a, b64, bstride);
  if (grid_out) *grid_out = (int)grid;
  return cudaGetLastError();
}

// Kept for the callers that ask whether the shared-memory FP64 kernels cover
// (N, k): they always do (up to 32 lanes per nplet).
int f64s_threads(int N, int k, size_t* smem_out) {
  const F64Cfg c = f64_config(N, k);
  if (smem_out) *smem_out = c.smem;
  return F64_NT / c.G;
}

// mode 0: five measures per nplet (SoA, per opt.out_f64); mode 2: basis
// values into b64 (3 arrays of bstride doubles, indexed by rank offset for
// the dense launch and by list position for the list launch).
cudaError_t launch_nplet_f64s(const NpletArgs& a, bool list, double* b64,
                              unsigned long long bstride, int num_sms, cudaStream_t s,
                              int* grid_out, int max_blocks) {
  const F64Cfg c = f64_config(a.N, a.k);
#define F64_CASE(GG)                                                                          \
  case GG:                                                                                    \
    return list ? launch_f64s_t<GG, true>(a, b64, bstride, c.smem, num_sms, s, grid_out,      \
                                          max_blocks)                                         \
                : launch_f64s_t<GG, false>(a, b64, bstride, c.smem, num_sms, s, grid_out,     \
                                           max_blocks);
  switch (c.G) {
    F64_CASE(1) F64_CASE(2) F64_CASE(4) F64_CASE(8) F64_CASE(16) F64_CASE(32)
    default: return cudaErrorInvalidValue;
  }
#undef F64_CASE
}

}  // namespace thoi
