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

// Starting thresholds of the top-M buffers: the M-th largest and the M-th
// smallest O of a sample of the range (SEED_RUNS runs of SEED_RUN
// consecutive elements, evenly spaced).  The M-th best of any subset is no
// better than the M-th best of the whole set, so every element of the true
// top M still passes; started near their final values, the reduction blocks
// see few candidates and sort little.  The M-th best is found by a radix
// select on order-preserving integer keys: a histogram of the top 11 bits
// picks the bin holding it, a histogram of the next 11 bits inside that bin
// narrows it, and the lower edge of that 22-bit bin (at least M samples at
// or above it) is the bound.
constexpr int SEED_NT = 1024;
constexpr int SEED_RUN = 256;
constexpr int SEED_RUNS = 512;
constexpr int SEED_S = SEED_RUN * SEED_RUNS;  // 131072 sampled elements
constexpr int SEED_BINS = 2048;

__device__ __forceinline__ unsigned fkey(float v) {
  unsigned u = __float_as_uint(v);
  if ((u << 1) == 0) u = 0;
  return (u >> 31) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_value(unsigned k) {
  return __uint_as_float((k >> 31) ? (k & 0x7fffffffu) : ~k);
}

// Bin (counting from the top) in which the running count of a descending
// scan of hist[SEED_BINS] reaches target; *above = count of the bins above
// it.  Run by warp 0.
__device__ void seed_find_bin(const unsigned* hist, unsigned target, int* bin, unsigned* above) {
  const int lane = threadIdx.x & 31;
  constexpr int PER = SEED_BINS / 32;
  // lane l owns bins [SEED_BINS - (l+1) PER, SEED_BINS - l PER), top first
  const int hi = SEED_BINS - lane * PER;
  unsigned mine = 0;
  for (int b = hi - 1; b >= hi - PER; b--) mine += hist[b];
  unsigned incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  const unsigned excl = incl - mine;
  const bool here = excl < target && incl >= target;
  const unsigned who = __ballot_sync(0xffffffffu, here);
  if (who == 0) {
    if (lane == 0) {
      *bin = -1;
      *above = 0;
    }
    return;
  }
  if (lane == __ffs(who) - 1) {
    unsigned run = excl;
    for (int b = hi - 1; b >= hi - PER; b--) {
      if (run + hist[b] >= target) {
        *bin = b;
        *above = run;
        break;
      }
      run += hist[b];
    }
  }
}

// Histogram increment aggregated over the lanes of a warp that hit the same
// bin (neighbouring samples usually share their high key bits, so one atomic
// per distinct bin replaces up to 32 on one address).
__device__ __forceinline__ void hist_add(unsigned* hist, unsigned bin, bool on) {
  const unsigned act = __ballot_sync(0xffffffffu, on);
  if (!on) return;
  const unsigned peers = __match_any_sync(act, bin);
  if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[bin], (unsigned)__popc(peers));
}

__global__ void __launch_bounds__(SEED_NT) k_seed_thresholds(const float* __restrict__ blr,
                                                             const float* __restrict__ bsp,
                                                             unsigned long long n, Combine cmb,
                                                             int top_m, float* __restrict__ thr) {
  __shared__ unsigned h[2][SEED_BINS];
  __shared__ int s_bin[2];
  __shared__ unsigned s_above[2];
  __shared__ unsigned s_valid;
  const CombineV<float> c(cmb);
  const unsigned long long S = n < (unsigned long long)SEED_S ? n : (unsigned long long)SEED_S;
  // Samples are read SEED_ILP at a time, all loads issued before any is used:
  // one block walks the whole sample, so the loop is bound by memory latency
  // unless many loads are in flight per thread.  Every lane of a warp runs the
  // same iterations (absent samples take part with on = false), as hist_add
  // needs.
  constexpr int SEED_ILP = 8;
  __shared__ unsigned long long s_run[SEED_RUNS];  // first element of each sampled run
  for (int r = threadIdx.x; r < SEED_RUNS; r += SEED_NT)
    s_run[r] = n > (unsigned long long)SEED_S
                   ? (unsigned long long)r * (n - SEED_RUN) / (SEED_RUNS - 1) : 0ull;
  __syncthreads();
  const int iters = ((int)S + SEED_NT * SEED_ILP - 1) / (SEED_NT * SEED_ILP);
  auto load_group = [&](int i0, float (&lr)[SEED_ILP], float (&sp)[SEED_ILP]) {
#pragma unroll
    for (int j = 0; j < SEED_ILP; j++) {
      const int q = threadIdx.x + (i0 * SEED_ILP + j) * SEED_NT;
      lr[j] = pinf<float>() - pinf<float>();
      sp[j] = 0.f;
      if (q < (int)S) {
        const unsigned long long e =
            n <= (unsigned long long)SEED_S ? (unsigned long long)q : s_run[q / SEED_RUN] + q % SEED_RUN;
        lr[j] = blr[e];
        sp[j] = bsp[e];
      }
    }
  };
  // order-preserving keys: largest O = largest kh; smallest O = largest kl
  auto keys_of = [&](float lr, float sp, unsigned& kh, unsigned& kl) -> bool {
    if (is_nan(lr)) return false;
    float v[5];
    combine5<float>(lr, sp, 0.f, c, v);  // the ranked measure (H would need the log-variances)
    kh = fkey(pick5(v, cmb.top));
    kl = ~kh;
    return true;
  };
  for (int q = threadIdx.x; q < 2 * SEED_BINS; q += SEED_NT) (&h[0][0])[q] = 0;
  if (threadIdx.x == 0) s_valid = 0;
  __syncthreads();
  unsigned valid = 0;
  for (int i0 = 0; i0 < iters; i0++) {
    float lr[SEED_ILP], sp[SEED_ILP];
    load_group(i0, lr, sp);
#pragma unroll
    for (int j = 0; j < SEED_ILP; j++) {
      unsigned kh = 0, kl = 0;
      const bool on = keys_of(lr[j], sp[j], kh, kl);
      valid += on ? 1u : 0u;
      hist_add(h[0], kh >> 21, on);
      hist_add(h[1], kl >> 21, on);
    }
  }
  atomicAdd(&s_valid, valid);
  __syncthreads();
  const unsigned M = (unsigned)top_m;
  if (threadIdx.x < 32) {
    seed_find_bin(h[0], M, &s_bin[0], &s_above[0]);
    seed_find_bin(h[1], M, &s_bin[1], &s_above[1]);
  }
  __syncthreads();
  const int b0 = s_bin[0], b1 = s_bin[1];
  const unsigned a0 = s_above[0], a1 = s_above[1];
  __syncthreads();
  for (int q = threadIdx.x; q < 2 * SEED_BINS; q += SEED_NT) (&h[0][0])[q] = 0;
  __syncthreads();
  if (s_valid >= M && b0 >= 0 && b1 >= 0) {
    for (int i0 = 0; i0 < iters; i0++) {
      float lr[SEED_ILP], sp[SEED_ILP];
      load_group(i0, lr, sp);
#pragma unroll
      for (int j = 0; j < SEED_ILP; j++) {
        unsigned kh = 0, kl = 0;
        const bool on = keys_of(lr[j], sp[j], kh, kl);
        hist_add(h[0], (kh >> 10) & (SEED_BINS - 1), on && (int)(kh >> 21) == b0);
        hist_add(h[1], (kl >> 10) & (SEED_BINS - 1), on && (int)(kl >> 21) == b1);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    if (s_valid >= M && b0 >= 0 && b1 >= 0) {
      seed_find_bin(h[0], M - a0, &s_bin[0], &s_above[0]);
      seed_find_bin(h[1], M - a1, &s_bin[1], &s_above[1]);
    } else if (threadIdx.x == 0) {
      s_bin[0] = s_bin[1] = -1;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // lower edges of the 22-bit bins (at least M samples at or above each),
    // widened by a relative 1e-6 so that a rounding difference between two
    // evaluations of O can never reject a top-M element
    if (s_bin[0] >= 0 && s_bin[1] >= 0) {
      const unsigned kh = ((unsigned)b0 << 21) | ((unsigned)s_bin[0] << 10);
      const unsigned kl = ((unsigned)b1 << 21) | ((unsigned)s_bin[1] << 10);
      const float hi = fkey_value(kh), lo = fkey_value(~kl);
      thr[0] = hi - 1e-6f * fabsf(hi) - 1e-30f;  // M-th largest (bound)
      thr[1] = lo + 1e-6f * fabsf(lo) + 1e-30f;  // M-th smallest (bound)
    } else {
      thr[0] = -pinf<float>();
      thr[1] = pinf<float>();
    }
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

// Candidate list of a fused-records order slot: block s reduces segment s
// of the list (the FP32 list reduction), seeded with the slot's top-list
// bounds (every nplet of the final top lists lies beyond them once the merge
// certifies the record).  The partials carry the extremes and the top lists
// only: the sums and the count of O < 0 came from the nplet kernel, and
// block 0 carries the count of FP32 nplets (the rank range less the nplets
// flagged for the FP64 re-factor).
__global__ void __launch_bounds__(RED_NT, 6) k_reduce_candidates(
    const float* __restrict__ cb, unsigned long long cap, unsigned long long seg,
    const unsigned long long* __restrict__ ids, const unsigned long long* cand_count,
    const unsigned* __restrict__ keys, Combine cmb, int top_m, unsigned long long n_range,
    const unsigned long long* flag_count, unsigned long long flag_cap, PartRec* __restrict__ part,
    TopEnt* __restrict__ part_top) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ RedScratch sc;
  __shared__ int s_tcnt[2];
  __shared__ float s_seed[2];
  if (threadIdx.x == 0) {
    s_seed[0] = fused_threshold(keys[5 + cmb.top], 5 + cmb.top, cmb.top);
    s_seed[1] = fused_threshold(keys[cmb.top], cmb.top, cmb.top);
  }
  __syncthreads();
  const unsigned long long o = (unsigned long long)blockIdx.x * seg;
  reduce_core<float, true>(threadIdx.x, RED_NT, cb + o, cb + cap + o, cb + 2 * cap + o, 0,
                           ids + o, cand_count + blockIdx.x, seg, 0, cmb, top_m, 0, s_seed,
                           part + blockIdx.x, part_top + (size_t)blockIdx.x * 2 * top_m, smem,
                           sc, s_tcnt, 2654435761ull);
  if (threadIdx.x == 0) {
    // same thread as the partial's writer in reduce_core
    PartRec* r = part + blockIdx.x;
    const unsigned long long fc = *flag_count;
    r->s_lr = r->s_sp = r->s_ls = 0.0;
    r->neg = 0;
    r->notpd = 0;
    r->count = blockIdx.x == 0 ? n_range - (fc < flag_cap ? fc : flag_cap) : 0ull;
  }
}

cudaError_t launch_reduce_candidates(const NpletArgs& a, int num_sms, int max_blocks,
                                     PartRec* part, TopEnt* part_top, cudaStream_t s,
                                     int* grid_out) {
  (void)num_sms;
  const size_t sm =
      a.top_m > 0 ? (size_t)RTOP_CAP * 2 * (sizeof(float) + sizeof(unsigned long long)) : 0;
  int occ = 0;
  cudaError_t e = occupancy_cached((const void*)k_reduce_candidates, RED_NT, sm, &occ);
  if (e != cudaSuccess) return e;
  if (a.cand_nseg < 1 || a.cand_nseg > max_blocks) return cudaErrorInvalidValue;
  k_reduce_candidates<<<(unsigned)a.cand_nseg, RED_NT, sm, s>>>(
      a.cand_b, a.cand_cap, a.cand_seg, a.cand_ids, a.cand_count, a.thr_keys, a.cmb, a.top_m,
      a.rank_end - a.rank_begin, a.flag_count, a.flag_cap, part, part_top);
  if (grid_out) *grid_out = a.cand_nseg;
  return cudaGetLastError();
}

cudaError_t launch_reduce_basis(const float* basis, unsigned long long stride_elems,
                                unsigned long long n, unsigned long long id0, Combine cmb,
                                int top_m, float* seed_thr, PartRec* part, TopEnt* part_top,
                                int num_sms, int max_blocks, cudaStream_t s, int* grid_out) {
  const float* thr = nullptr;
  // the seed samples do not read the log-variances, so H-ranked lists start unseeded
  if (top_m > 0 && seed_thr && n > (1ull << 20) && cmb.top != THOI_H) {
    k_seed_thresholds<<<1, SEED_NT, 0, s>>>(basis, basis + stride_elems, n, cmb, top_m, seed_thr);
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
