// Streaming per-order reduction of the FP32 path.  The nplet kernels write
// three basis values per nplet (log det R_S, sum_j log p_j, sum_i log
// Sigma_ii; NaN log det = re-factored in FP64); this kernel reads them
// back (coalesced, 16-byte loads), forms the five measures and reduces them
// per block: min/max with the smallest id on ties, sums, counts, count of
// O < 0 and the top-M lists (Fig. 1A caption: a function applied to every
// batch, here a fixed reduction set).  Keeping the reduction out of the
// compute kernels frees their registers and removes their barriers.
#include "nplet_common.cuh"

namespace thoi {

constexpr int RB_PER_THREAD = 4;  // elements per thread per round (one float4 of each array)

__global__ void __launch_bounds__(RED_NT) k_reduce_basis(const float* __restrict__ blr,
                                                         const float* __restrict__ bsp,
                                                         const float* __restrict__ bls,
                                                         unsigned long long n,
                                                         unsigned long long id0, Combine cmb,
                                                         int top_m, PartRec* __restrict__ part,
                                                         TopEnt* __restrict__ part_top) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ RedScratch sc;
  __shared__ int s_tcnt[2];
  const bool with_top = top_m > 0;
  TopBuf<float, unsigned> tb;
  tb.val[0] = reinterpret_cast<float*>(smem);
  tb.val[1] = tb.val[0] + TOP_CAP;
  tb.idx[0] = reinterpret_cast<unsigned*>(tb.val[1] + TOP_CAP);
  tb.idx[1] = tb.idx[0] + TOP_CAP;
  tb.cnt = s_tcnt;
  if (threadIdx.x == 0) s_tcnt[0] = s_tcnt[1] = 0;
  __syncthreads();
  float thr_hi = -pinf<float>(), thr_lo = pinf<float>();
  ThreadRed<float, unsigned> tr;
  tr.init();
  const unsigned long long nq = (n + RB_PER_THREAD - 1) / RB_PER_THREAD;
  const unsigned long long stride = (unsigned long long)gridDim.x * RED_NT;
  const unsigned long long rounds = (nq + stride - 1) / stride;
  const int trigger = TOP_CAP - RED_NT * RB_PER_THREAD;
  for (unsigned long long rd = 0; rd < rounds; rd++) {
    const unsigned long long q = rd * stride + (unsigned long long)blockIdx.x * RED_NT + threadIdx.x;
    if (q < nq) {
      const unsigned long long e0 = q * RB_PER_THREAD;
      float lr[4], sp[4], ls[4];
      if (e0 + 4 <= n) {
        const float4 x = reinterpret_cast<const float4*>(blr)[q];
        const float4 y = reinterpret_cast<const float4*>(bsp)[q];
        const float4 z = reinterpret_cast<const float4*>(bls)[q];
        lr[0] = x.x; lr[1] = x.y; lr[2] = x.z; lr[3] = x.w;
        sp[0] = y.x; sp[1] = y.y; sp[2] = y.z; sp[3] = y.w;
        ls[0] = z.x; ls[1] = z.y; ls[2] = z.z; ls[3] = z.w;
      } else {
#pragma unroll
        for (int t = 0; t < 4; t++) {
          const bool ok = e0 + t < n;
          lr[t] = ok ? blr[e0 + t] : __int_as_float(0x7fc00000);
          sp[t] = ok ? bsp[e0 + t] : 0.f;
          ls[t] = ok ? bls[e0 + t] : 0.f;
        }
      }
#pragma unroll
      for (int t = 0; t < 4; t++) {
        if (isnan(lr[t])) continue;  // re-factored in FP64, or past the end
        float v[5];
        combine5<float>(lr[t], sp[t], ls[t], cmb, v);
        const unsigned loc = (unsigned)(e0 + t);
        tr.add(v, loc, lr[t], sp[t], ls[t]);
        if (with_top) top_offer(tb, v[3], loc, thr_hi, thr_lo);
      }
      tr.flush();
    }
    if (with_top) {
      __syncthreads();
      const bool c0 = tb.cnt[0] > trigger, c1 = tb.cnt[1] > trigger;
      if (c0) {
        top_sort_cut(tb, 0, top_m);
        thr_hi = top_threshold(tb, 0, top_m);
      }
      if (c1) {
        top_sort_cut(tb, 1, top_m);
        thr_lo = top_threshold(tb, 1, top_m);
      }
      __syncthreads();
    }
  }
  int th = 0, tl = 0;
  if (with_top) {
    top_sort_cut(tb, 0, top_m);
    top_sort_cut(tb, 1, top_m);
    th = tb.cnt[0];
    tl = tb.cnt[1];
    top_write(tb, top_m, id0, part_top + (size_t)blockIdx.x * 2 * top_m);
  }
  block_write_part<float, unsigned>(tr, 0u, id0, sc, part + blockIdx.x, th, tl);
}

cudaError_t launch_reduce_basis(const float* basis, unsigned long long stride_elems,
                                unsigned long long n, unsigned long long id0, Combine cmb,
                                int top_m, PartRec* part, TopEnt* part_top, int num_sms,
                                int max_blocks, cudaStream_t s, int* grid_out) {
  const size_t sm = top_m > 0 ? (size_t)TOP_CAP * 2 * (sizeof(float) + sizeof(unsigned)) : 0;
  cudaError_t e = cudaFuncSetAttribute(k_reduce_basis, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_reduce_basis, RED_NT, sm);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  long long grid = (long long)num_sms * occ;
  const long long need = (long long)((n + RED_NT * RB_PER_THREAD - 1) / (RED_NT * RB_PER_THREAD));
  if (need < grid) grid = need > 0 ? need : 1;
  if (grid > max_blocks) grid = max_blocks;
  k_reduce_basis<<<(unsigned)grid, RED_NT, sm, s>>>(basis, basis + stride_elems,
                                                    basis + 2 * stride_elems, n, id0, cmb, top_m,
                                                    part, part_top);
  if (grid_out) *grid_out = (int)grid;
  return cudaGetLastError();
}

}  // namespace thoi
