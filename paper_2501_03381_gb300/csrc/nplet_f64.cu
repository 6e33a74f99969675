// FP64 nplet kernel: the THOI_F64 path and the re-factor of the nplets the
// FP32 path flagged.  One nplet per thread; each thread's k x k matrix lives
// in shared memory, interleaved across the block (entry e of thread t at
// mat[e * NT + t], so a warp's accesses to "its" entry are consecutive).
// FP64 arithmetic runs at a small fraction of the FP32 rate on this GPU, so
// shared-memory bandwidth is ample; what matters is latency, and shared
// memory keeps it far below that of per-thread local arrays.
//
// Same quantities as the FP32 kernels: R_S = Lh D Lh^T, log det R_S =
// sum log D_p, the unit-lower inverse V column by column, and
// p_j = (R_S^-1)_jj = 1/D_j + sum_{i>j} V_ij^2 / D_i.  A pivot D_p <= 0 marks
// the nplet not positive definite.
#include "nplet_f64.cuh"

namespace thoi {

template <int NT, bool LIST, typename M>
__global__ void __launch_bounds__(NT) k_nplet_f64s(const NpletArgs a, double* __restrict__ b64,
                                                   unsigned long long bstride) {
  extern __shared__ __align__(16) unsigned char smem[];
  f64s_body<NT, LIST, M>(a, b64, bstride, smem);
}

template <int NT, bool LIST>
static cudaError_t launch_f64s_t(const NpletArgs& a, double* b64, unsigned long long bstride,
                                 size_t sm, int num_sms, cudaStream_t s, int* grid_out,
                                 int max_blocks) {
  void (*fn)(const NpletArgs, double*, unsigned long long);
  if (a.N > 32) fn = k_nplet_f64s<NT, LIST, unsigned long long>;
  else fn = k_nplet_f64s<NT, LIST, unsigned>;
  int occ = 0;
  cudaError_t e = occupancy_cached((const void*)fn, NT, sm, &occ);
  if (e != cudaSuccess) return e;
  long long grid = (long long)num_sms * occ;
  if (!LIST) {
    const unsigned long long n = a.rank_end - a.rank_begin;
    const long long need = (long long)((n + NT - 1) / NT);
    if (need < grid) grid = need > 0 ? need : 1;
  }
  if (grid > max_blocks) grid = max_blocks;
  fn<<<(unsigned)grid, NT, sm, s>>>(a, b64, bstride);
  if (grid_out) *grid_out = (int)grid;
  return cudaGetLastError();
}

// Threads per block so that the block's matrices fit in shared memory; 0 if
// even 32 matrices do not fit (the caller then uses the generic kernel).
int f64s_threads(int N, int k, size_t* smem_out) {
  const SmemLayout L = smem_layout(N, k, row_stride(N), sizeof(double), 8, 0);
  const size_t per = (size_t)(k * (k + 1) / 2) * sizeof(double);
  const size_t budget = 220 * 1024;
  for (int nt = 128; nt >= 32; nt >>= 1) {
    const size_t sm = L.total + per * nt;
    if (sm <= budget) {
      if (smem_out) *smem_out = sm;
      return nt;
    }
  }
  return 0;
}

// mode 0: five measures per nplet (SoA, per opt.out_f64); mode 2: basis
// values into b64 (3 arrays of bstride doubles, indexed by rank offset for
// the dense launch and by list position for the list launch).
cudaError_t launch_nplet_f64s(const NpletArgs& a, bool list, double* b64,
                              unsigned long long bstride, int num_sms, cudaStream_t s,
                              int* grid_out, int max_blocks) {
  size_t sm = 0;
  const int nt = f64s_threads(a.N, a.k, &sm);
  if (nt == 0) return cudaErrorInvalidValue;
  if (list) {
    if (nt == 128) return launch_f64s_t<128, true>(a, b64, bstride, sm, num_sms, s, grid_out, max_blocks);
    if (nt == 64) return launch_f64s_t<64, true>(a, b64, bstride, sm, num_sms, s, grid_out, max_blocks);
    return launch_f64s_t<32, true>(a, b64, bstride, sm, num_sms, s, grid_out, max_blocks);
  }
  if (nt == 128) return launch_f64s_t<128, false>(a, b64, bstride, sm, num_sms, s, grid_out, max_blocks);
  if (nt == 64) return launch_f64s_t<64, false>(a, b64, bstride, sm, num_sms, s, grid_out, max_blocks);
  return launch_f64s_t<32, false>(a, b64, bstride, sm, num_sms, s, grid_out, max_blocks);
}

}  // namespace thoi
