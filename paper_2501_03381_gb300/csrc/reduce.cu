// Streaming per-order reduction.  The nplet kernels write three basis values
// per nplet (log det R_S, sum_j log p_j, sum_i log Sigma_ii; a NaN log det
// marks a nplet that is reduced elsewhere or is not positive definite); this
// kernel reads them back, forms the five measures and reduces them per block:
// min/max with the smallest id on ties, sums, counts, count of O < 0 and the
// top-M lists (Fig. 1A caption: a function applied to every batch, here a
// fixed reduction set).  Keeping the reduction out of the compute kernels
// frees their registers and removes their barriers.
//
// Instances: FP32 values with dense ids (the FP32 path; NaN = re-factored in
// FP64, skipped), FP64 values with dense ids (the FP64 path; NaN = not
// positive definite) and FP64 values with ids from the re-factor list.
#include "reduce.cuh"

namespace thoi {

// Starting thresholds of the top-M buffers: the M-th largest and M-th
// smallest O among a sample of the elements (SEED_CHUNKS runs of SEED_RUN
// consecutive elements spread over the range).  The M-th best of any subset
// is no better than the M-th best of the whole set, so every element of the
// true top-M still passes; with the thresholds starting near their final
// values, the blocks see few candidates and rarely compact.
constexpr int SEED_NT = 1024;
constexpr int SEED_CHUNKS = 64;
constexpr int SEED_RUN = 256;
constexpr int SEED_S = SEED_CHUNKS * SEED_RUN;  // 16384 sampled elements

__global__ void __launch_bounds__(SEED_NT) k_seed_thresholds(const float* __restrict__ blr,
                                                             const float* __restrict__ bsp,
                                                             unsigned long long n, Combine cmb,
                                                             int top_m, float* __restrict__ thr) {
  extern __shared__ __align__(16) float sv[];  // SEED_S values
  __shared__ int s_valid;
  const CombineV<float> c(cmb);
  if (threadIdx.x == 0) s_valid = 0;
  __syncthreads();
  const unsigned long long S = n < (unsigned long long)SEED_S ? n : (unsigned long long)SEED_S;
  int valid = 0;
  for (int q = threadIdx.x; q < SEED_S; q += SEED_NT) {
    float o = pinf<float>();
    if ((unsigned long long)q < S) {
      unsigned long long e;
      if (n <= (unsigned long long)SEED_S) {
        e = q;
      } else {
        const int ch = q / SEED_RUN, off = q % SEED_RUN;
        e = (unsigned long long)ch * (n - SEED_RUN) / (SEED_CHUNKS - 1) + off;
      }
      const float lr = blr[e];
      if (!is_nan(lr)) {
        const float sp = bsp[e];
        const float tc = -0.5f * lr + c.tc_c, dtc = 0.5f * (lr + sp) + c.dtc_c;
        o = tc - dtc;
        valid++;
      }
    }
    sv[q] = o;  // invalid -> +inf, sorted to the end
  }
  atomicAdd(&s_valid, valid);
  __syncthreads();
  for (int kk = 2; kk <= SEED_S; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < SEED_S; i += SEED_NT) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const bool up = (i & kk) == 0;
          const float x = sv[i], y = sv[ixj];
          if (up ? (y < x) : (x < y)) { sv[i] = y; sv[ixj] = x; }
        }
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    // widened by a relative 1e-6 so that a rounding difference between this
    // kernel's O and the reduction's O can never reject a top-M element
    const int V = s_valid;
    const float hi = sv[V >= top_m ? V - top_m : 0], lo = sv[top_m - 1 < SEED_S ? top_m - 1 : 0];
    thr[0] = V >= top_m ? hi - 1e-6f * fabsf(hi) - 1e-30f : -pinf<float>();  // M-th largest
    thr[1] = V >= top_m ? lo + 1e-6f * fabsf(lo) + 1e-30f : pinf<float>();   // M-th smallest
  }
}

template <typename V, bool LIST>
__global__ void __launch_bounds__(RED_NT, 6) k_reduce_basis(
    const V* __restrict__ blr, const V* __restrict__ bsp, const V* __restrict__ bls,
    unsigned long long n_dense, const unsigned long long* __restrict__ ids,
    const unsigned long long* list_count, unsigned long long list_cap, unsigned long long id0,
    Combine cmb, int top_m, int nan_is_notpd, const float* __restrict__ seed_thr,
    PartRec* __restrict__ part, TopEnt* __restrict__ part_top) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ RedScratch sc;
  __shared__ int s_tcnt[2];
  reduce_core<V, LIST>((unsigned long long)blockIdx.x * RED_NT + threadIdx.x,
                       (unsigned long long)gridDim.x * RED_NT, blr, bsp, bls, n_dense, ids,
                       list_count, list_cap, id0, cmb, top_m, nan_is_notpd, seed_thr,
                       part + blockIdx.x, part_top + (size_t)blockIdx.x * 2 * top_m, smem, sc,
                       s_tcnt);
}

template <typename V, bool LIST>
static cudaError_t launch_reduce_t(const V* basis, unsigned long long stride_elems,
                                   unsigned long long n, const unsigned long long* ids,
                                   const unsigned long long* list_count,
                                   unsigned long long list_cap, unsigned long long id0, Combine cmb,
                                   int top_m, int nan_is_notpd, const float* seed_thr,
                                   PartRec* part, TopEnt* part_top, int num_sms, int max_blocks,
                                   cudaStream_t s, int* grid_out) {
  using I = typename std::conditional<LIST, unsigned long long, unsigned>::type;
  const size_t sm = top_m > 0 ? (size_t)RTOP_CAP * 2 * (sizeof(V) + sizeof(I)) : 0;
  void (*fn)(const V*, const V*, const V*, unsigned long long, const unsigned long long*,
             const unsigned long long*, unsigned long long, unsigned long long, Combine, int, int,
             const float*, PartRec*, TopEnt*) = k_reduce_basis<V, LIST>;
  int occ = 0;
  cudaError_t e = occupancy_cached((const void*)fn, RED_NT, sm, &occ);
  if (e != cudaSuccess) return e;
  long long grid = (long long)num_sms * occ;
  if (!LIST) {
    const long long need =
        (long long)((n + RED_NT * RB_PER_THREAD - 1) / (RED_NT * RB_PER_THREAD));
    if (need < grid) grid = need > 0 ? need : 1;
  }
  if (grid > max_blocks) grid = max_blocks;
  fn<<<(unsigned)grid, RED_NT, sm, s>>>(basis, basis + stride_elems, basis + 2 * stride_elems, n,
                                        ids, list_count, list_cap, id0, cmb, top_m, nan_is_notpd,
                                        seed_thr, part, part_top);
  if (grid_out) *grid_out = (int)grid;
  return cudaGetLastError();
}

cudaError_t launch_reduce_basis(const float* basis, unsigned long long stride_elems,
                                unsigned long long n, unsigned long long id0, Combine cmb,
                                int top_m, float* seed_thr, PartRec* part, TopEnt* part_top,
                                int num_sms, int max_blocks, cudaStream_t s, int* grid_out) {
  const float* thr = nullptr;
  if (top_m > 0 && seed_thr && n > (8ull << 20)) {
    const size_t sm = (size_t)SEED_S * sizeof(float);
    int occ = 0;
    cudaError_t e = occupancy_cached((const void*)k_seed_thresholds, SEED_NT, sm, &occ);
    if (e != cudaSuccess) return e;
    k_seed_thresholds<<<1, SEED_NT, sm, s>>>(basis, basis + stride_elems, n, cmb, top_m, seed_thr);
    thr = seed_thr;
  }
  return launch_reduce_t<float, false>(basis, stride_elems, n, nullptr, nullptr, 0, id0, cmb, top_m,
                                       0, thr, part, part_top, num_sms, max_blocks, s, grid_out);
}

cudaError_t launch_reduce_basis64(const double* basis, unsigned long long stride_elems,
                                  unsigned long long n, unsigned long long id0, Combine cmb,
                                  int top_m, PartRec* part, TopEnt* part_top, int num_sms,
                                  int max_blocks, cudaStream_t s, int* grid_out) {
  return launch_reduce_t<double, false>(basis, stride_elems, n, nullptr, nullptr, 0, id0, cmb,
                                        top_m, 1, nullptr, part, part_top, num_sms, max_blocks, s,
                                        grid_out);
}

cudaError_t launch_reduce_list64(const double* basis, unsigned long long stride_elems,
                                 const unsigned long long* ids, const unsigned long long* count,
                                 unsigned long long cap, Combine cmb, int top_m, PartRec* part,
                                 TopEnt* part_top, int num_sms, int max_blocks, cudaStream_t s,
                                 int* grid_out) {
  return launch_reduce_t<double, true>(basis, stride_elems, 0, ids, count, cap, 0, cmb, top_m, 1,
                                       nullptr, part, part_top, num_sms, max_blocks, s, grid_out);
}

}  // namespace thoi
