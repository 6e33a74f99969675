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
#include <cstring>

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

constexpr unsigned long long RED_MIN_PER_BLOCK = 1ull << 14;

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
    // at least 16K elements per block: a short range in many blocks would
    // leave the merge many top lists of few entries each to sift
    const long long need = (long long)((n + RED_MIN_PER_BLOCK - 1) / RED_MIN_PER_BLOCK);
    if (need < grid) grid = need > 0 ? need : 1;
  }
  if (grid > max_blocks) grid = max_blocks;
  fn<<<(unsigned)grid, RED_NT, sm, s>>>(basis, basis + stride_elems, basis + 2 * stride_elems, n,
                                        ids, list_count, list_cap, id0, cmb, top_m, nan_is_notpd,
                                        seed_thr, part, part_top);
  if (grid_out) *grid_out = (int)grid;
  return cudaGetLastError();
}

// Radix-select reductions.  A source is a list of basis-value triples in
// one or more segments: the candidate list of a fused-records order slot
// (see nplet_common.cuh; FP32, explicit ids, 16 segments with device
// counts), a dense range of FP32 basis values (ids from the position), or
// an FP64 re-factor list (explicit ids, device count).  One streaming pass
// gives the extremes of every measure, the sums and counts, and a
// histogram of the top 11 bits of the order-preserving key of the ranked
// measure (rounded to FP32: the rounding is monotone, so the key order
// never contradicts the value order); the bin holding the M-th best, a
// histogram of the next 11 bits inside it, then every entry at or beyond
// the 22-bit bin so found (the top M and the few tied with them to 2^-13
// relative) is gathered and sorted by value, then id.  No per-block top
// buffers are cut and recut, whatever the order of the list.
// Partials: SEL_SUB blocks (or the launch's count) per segment carry the
// record fields, then one partial carries the two top lists.
constexpr int CAND_SUB = 48;       // blocks per candidate segment
constexpr int SEL_SURV = 8192;     // gathered entries per side, at most
constexpr int CAND_BINS = 2048;
constexpr size_t CW_HIST1 = 0;
constexpr size_t CW_HIST2 = CW_HIST1 + 2 * CAND_BINS * 4;
constexpr size_t CW_SEL = CW_HIST2 + 2 * CAND_BINS * 4;   // bin1[2], above1[2], bin2[2], above2[2], n[2]
constexpr size_t CW_HEAD = CW_SEL + 256;                    // zeroed per slot
constexpr size_t CW_SV = CW_HEAD;                           // value [2][SEL_SURV] (8 B slots)
constexpr size_t CW_SI = CW_SV + 2 * SEL_SURV * 8;          // u64 [2][SEL_SURV]
constexpr size_t CW_BYTES = CW_SI + 2 * SEL_SURV * 8;
constexpr unsigned long long SEL_PER_BLOCK = 8192;  // dense ranges: entries per pass block
constexpr int SEL_LIST_BLOCKS = 48;                 // re-factor lists: pass blocks

size_t cand_ws_bytes() { return CW_BYTES; }
size_t sel_ws_bytes() { return CW_BYTES; }
int cand_partials(int nseg) { return nseg * CAND_SUB + 1; }

// One source of a select reduction.
struct SelSrc {
  const void* basis;                 // V: lr at [p], sp at [stride + p], lsum at [2 stride + p]
  unsigned long long stride;
  const unsigned long long* ids;     // id of entry p; null: id0 + p
  unsigned long long id0;
  const unsigned long long* counts;  // entries of each segment (device); null: n each
  unsigned long long n;              // entries, or the capacity of a segment
  unsigned long long seg_len;        // entry e of segment s sits at s * seg_len + e
  int nseg;
  int nan_notpd;                     // a NaN log det counts as not positive definite
  int fused;                         // candidate list: partial 0 carries the FP32 count
  unsigned long long rank_count;     // fused: ranks of the slot
  const unsigned long long* flag_count;
  unsigned long long flag_cap;
  Combine cmb;
  int top_m;
  int* status;
  unsigned char* ws;
};

__device__ __forceinline__ unsigned cand_key(float v, int side) {
  const unsigned k = fkey(v);
  return side == 0 ? k : ~k;
}

__device__ __forceinline__ unsigned long long sel_entries(const SelSrc& src, int seg) {
  if (!src.counts) return src.n;
  const unsigned long long c = src.counts[seg];
  return c < src.n ? c : src.n;
}

// pass 0: record fields, and the histogram of the top 11 key bits (both
// sides); pass 1: inside the selected top bins, the histogram of the next
// 11 bits; pass 2: gather the entries at or beyond the selected 22-bit bins.
template <typename V>
__global__ void __launch_bounds__(RED_NT) k_sel_pass(const SelSrc src, int pass,
                                                     PartRec* __restrict__ part) {
  __shared__ unsigned h[2][CAND_BINS];
  __shared__ RedScratch sc;
  const int seg = blockIdx.y;
  const unsigned long long n = sel_entries(src, seg);
  const unsigned long long base = (unsigned long long)seg * src.seg_len;
  const V* cb = static_cast<const V*>(src.basis);
  const CombineV<V> cv(src.cmb);
  const int top = src.cmb.top;
  unsigned char* ws = src.ws;
  unsigned* gh1 = reinterpret_cast<unsigned*>(ws + CW_HIST1);
  unsigned* gh2 = reinterpret_cast<unsigned*>(ws + CW_HIST2);
  unsigned* nsurv = reinterpret_cast<unsigned*>(ws + CW_SEL) + 8;
  V* sv = reinterpret_cast<V*>(ws + CW_SV);
  unsigned long long* si = reinterpret_cast<unsigned long long*>(ws + CW_SI);
  if (pass < 2) {
    for (int q = threadIdx.x; q < 2 * CAND_BINS; q += RED_NT) (&h[0][0])[q] = 0;
    __syncthreads();
  }
  ThreadRed<V, unsigned long long> tr;
  tr.init();
  unsigned notpd = 0;
  // the selected bins (pass 1) and 22-bit thresholds (pass 2), found by
  // every block from the finished histograms (warp w: side w); a bin of -1
  // means fewer than M entries on that side: everything is kept
  __shared__ int s_bin[4];
  __shared__ unsigned s_above[4];
  int b1[2] = {0, 0};
  unsigned t22[2] = {0u, 0u};
  if (pass >= 1) {
    if (threadIdx.x < 64) {
      const int sd = threadIdx.x >> 5;
      seed_find_bin(gh1 + sd * CAND_BINS, (unsigned)src.top_m, &s_bin[sd], &s_above[sd]);
      __syncwarp();
      if (pass == 2) {
        if (s_bin[sd] < 0) {
          if ((threadIdx.x & 31) == 0) s_bin[2 + sd] = -1;
        } else {
          seed_find_bin(gh2 + sd * CAND_BINS, (unsigned)src.top_m - s_above[sd], &s_bin[2 + sd],
                        &s_above[2 + sd]);
        }
      }
    }
    __syncthreads();
    for (int sd = 0; sd < 2; sd++) {
      b1[sd] = s_bin[sd];
      const int b2 = pass == 2 ? s_bin[2 + sd] : 0;
      t22[sd] = (b1[sd] < 0 || b2 < 0) ? 0u : (((unsigned)b1[sd] << 11) | (unsigned)b2);
    }
  }
  // every thread of a block runs the same rounds (the histogram increments
  // are aggregated over the lanes of a warp that hit the same bin: the
  // candidates crowd into the few bins near the bounds)
  for (unsigned long long e0 = (unsigned long long)blockIdx.x * RED_NT; e0 < n;
       e0 += (unsigned long long)gridDim.x * RED_NT) {
    const unsigned long long e = e0 + threadIdx.x;
    const unsigned long long p = base + e;
    bool ok = e < n;
    V lr = (V)0, sp = (V)0, ls = (V)0;
    if (ok) {
      lr = cb[p];
      sp = cb[src.stride + p];
      ls = cb[2 * src.stride + p];
      if (is_nan(lr)) {
        notpd += src.nan_notpd ? 1u : 0u;
        ok = false;
      }
    }
    V v[5];
    combine5<V>(lr, sp, ls, cv, v);
    const V o = pick5(v, top);
    const float fo = (float)o;
    const unsigned long long id = !ok ? 0ull : (src.ids ? src.ids[p] : src.id0 + p);
    if (pass == 0) {
      if (ok) tr.add(v, id, lr, sp, ls);
      if (src.top_m > 0) {
        hist_add(h[0], cand_key(fo, 0) >> 21, ok);
        hist_add(h[1], cand_key(fo, 1) >> 21, ok);
      }
    } else if (pass == 1) {
#pragma unroll
      for (int sd = 0; sd < 2; sd++) {
        const unsigned k = cand_key(fo, sd);
        hist_add(h[sd], (k >> 10) & 2047u, ok && b1[sd] >= 0 && (int)(k >> 21) == b1[sd]);
      }
    } else if (ok) {
#pragma unroll
      for (int sd = 0; sd < 2; sd++) {
        if ((cand_key(fo, sd) >> 10) >= t22[sd]) {
          const unsigned q = atomicAdd(&nsurv[sd], 1u);
          if (q < (unsigned)SEL_SURV) {
            sv[sd * SEL_SURV + q] = o;
            si[sd * SEL_SURV + q] = id;
          } else {
            atomicOr(src.status, ST_INEXACT);  // repeated with the streaming reductions
          }
        }
      }
    }
  }
  if (pass < 2) {
    __syncthreads();
    unsigned* g = pass == 0 ? gh1 : gh2;
    for (int q = threadIdx.x; q < 2 * CAND_BINS; q += RED_NT) {
      const unsigned c = (&h[0][0])[q];
      if (c) atomicAdd(&g[q], c);
    }
  }
  if (pass == 0) {
    const int pidx = seg * gridDim.x + blockIdx.x;
    block_write_part<V, unsigned long long>(tr, notpd, 0ull, sc, part + pidx, 0, 0);
    if (src.fused && threadIdx.x == 0) {
      // same thread as the partial's writer: the sums and the count of O < 0
      // come from the nplet kernel's partials, the count from the rank range
      PartRec* r = part + pidx;
      const unsigned long long fc = *src.flag_count;
      r->s_lr = r->s_sp = r->s_ls = 0.0;
      r->neg = 0;
      r->notpd = 0;
      r->count = pidx == 0 ? src.rank_count - (fc < src.flag_cap ? fc : src.flag_cap) : 0ull;
    }
  }
}

// The gathered entries of side blockIdx.x sorted best first (value, then the
// smaller id); the first M become the slot's top list.
template <typename V>
__global__ void __launch_bounds__(256) k_sel_final(const SelSrc src, PartRec* __restrict__ part,
                                                   TopEnt* __restrict__ part_top) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int sd = blockIdx.x;
  unsigned char* ws = src.ws;
  const unsigned* nsurv = reinterpret_cast<const unsigned*>(ws + CW_SEL) + 8;
  const V* sv = reinterpret_cast<const V*>(ws + CW_SV) + sd * SEL_SURV;
  const unsigned long long* si =
      reinterpret_cast<const unsigned long long*>(ws + CW_SI) + (size_t)sd * SEL_SURV;
  unsigned long long* idx = reinterpret_cast<unsigned long long*>(smem);
  V* val = reinterpret_cast<V*>(smem + SEL_SURV * 8);
  const int M = src.top_m;
  const int c = nsurv[sd] < (unsigned)SEL_SURV ? (int)nsurv[sd] : SEL_SURV;
  int P2 = 2;
  while (P2 < c) P2 <<= 1;
  const V sent = sd == 0 ? -pinf<V>() : pinf<V>();
  for (int q = threadIdx.x; q < P2; q += blockDim.x) {
    val[q] = q < c ? sv[q] : sent;
    idx[q] = q < c ? si[q] : ~0ull;
  }
  __syncthreads();
  for (int kk = 2; kk <= P2; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P2; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const bool up = (i & kk) == 0;
          const V vi = val[i], vj = val[ixj];
          const unsigned long long ii = idx[i], ij = idx[ixj];
          const bool sw = up ? top_before(sd, vj, ij, vi, ii) : top_before(sd, vi, ii, vj, ij);
          if (sw) {
            val[i] = vj; val[ixj] = vi;
            idx[i] = ij; idx[ixj] = ii;
          }
        }
      }
      __syncthreads();
    }
  }
  const int nout = c < M ? c : M;
  TopEnt* dst = part_top + (size_t)sd * M;
  for (int q = threadIdx.x; q < M; q += blockDim.x) {
    TopEnt e;
    if (q < nout) {
      e.v = (double)val[q];
      e.id = idx[q];
    } else {
      e.v = 0.0;
      e.id = ~0ull;
    }
    dst[q] = e;
  }
  if (threadIdx.x == 0) {
    // the two blocks write disjoint fields of the one partial
    if (sd == 0) {
      for (int m = 0; m < 5; m++) {
        part->vmin[m] = pinf<double>();
        part->vmax[m] = -pinf<double>();
        part->imin[m] = part->imax[m] = ~0ull;
      }
      part->s_lr = part->s_sp = part->s_ls = 0.0;
      part->count = part->neg = part->notpd = 0;
      part->top_hi = nout;
      if (gridDim.x == 1) part->top_lo = 0;
    } else {
      part->top_lo = nout;
    }
  }
}

// gx pass blocks per segment; partials: gx * nseg, then the top partial.
template <typename V>
static cudaError_t launch_select(const SelSrc& src, int gx, PartRec* part, TopEnt* part_top,
                                 cudaStream_t s, int* grid_out) {
  if (src.nseg < 1 || gx < 1 || !src.ws || !src.status) return cudaErrorInvalidValue;
  const int np = gx * src.nseg + 1;
  cudaError_t e = cudaMemsetAsync(src.ws, 0, CW_HEAD, s);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)gx, (unsigned)src.nseg);
  k_sel_pass<V><<<grid, RED_NT, 0, s>>>(src, 0, part);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  PartRec* ptop = part + np - 1;
  TopEnt* ttop = part_top ? part_top + (size_t)(np - 1) * 2 * src.top_m : nullptr;
  const size_t sm = (size_t)SEL_SURV * (8 + sizeof(V));
  static_assert((size_t)SEL_SURV * 16 <= 227 * 1024, "survivor sort exceeds shared memory");
  int occ = 0;
  if ((e = occupancy_cached((const void*)k_sel_final<V>, 256, sm, &occ)) != cudaSuccess) return e;
  if (src.top_m > 0) {
    k_sel_pass<V><<<grid, RED_NT, 0, s>>>(src, 1, part);
    k_sel_pass<V><<<grid, RED_NT, 0, s>>>(src, 2, part);
    k_sel_final<V><<<2, 256, sm, s>>>(src, ptop, ttop);
  } else {
    // an empty top partial (no lists)
    k_sel_final<V><<<1, 256, sm, s>>>(src, ptop, ttop);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (grid_out) *grid_out = np;
  return cudaSuccess;
}

cudaError_t launch_reduce_candidates(const NpletArgs& a, int num_sms, int max_blocks,
                                     PartRec* part, TopEnt* part_top, cudaStream_t s,
                                     int* grid_out) {
  (void)num_sms;
  if (a.cand_nseg < 1 || cand_partials(a.cand_nseg) > max_blocks) return cudaErrorInvalidValue;
  SelSrc src;
  memset(&src, 0, sizeof src);
  src.basis = a.cand_b;
  src.stride = a.cand_cap;
  src.ids = a.cand_ids;
  src.counts = a.cand_count;
  src.n = a.cand_seg;
  src.seg_len = a.cand_seg;
  src.nseg = a.cand_nseg;
  src.fused = 1;
  src.rank_count = a.rank_end - a.rank_begin;
  src.flag_count = a.flag_count;
  src.flag_cap = a.flag_cap;
  src.cmb = a.cmb;
  src.top_m = a.top_m;
  src.status = a.status;
  src.ws = a.cand_ws;
  return launch_select<float>(src, CAND_SUB, part, part_top, s, grid_out);
}

cudaError_t launch_select_basis(const float* basis, unsigned long long stride_elems,
                                unsigned long long n, unsigned long long id0, Combine cmb,
                                int top_m, unsigned char* ws, int* status, PartRec* part,
                                TopEnt* part_top, int max_blocks, cudaStream_t s, int* grid_out) {
  SelSrc src;
  memset(&src, 0, sizeof src);
  src.basis = basis;
  src.stride = stride_elems;
  src.id0 = id0;
  src.n = n;
  src.nseg = 1;
  src.cmb = cmb;
  src.top_m = top_m;
  src.status = status;
  src.ws = ws;
  long long gx = (long long)((n + SEL_PER_BLOCK - 1) / SEL_PER_BLOCK);
  if (gx < 1) gx = 1;
  if (gx > max_blocks - 1) gx = max_blocks - 1;
  if (gx < 1) return cudaErrorInvalidValue;
  return launch_select<float>(src, (int)gx, part, part_top, s, grid_out);
}

cudaError_t launch_select_basis64(const double* basis, unsigned long long stride_elems,
                                  unsigned long long n, unsigned long long id0, Combine cmb,
                                  int top_m, unsigned char* ws, int* status, PartRec* part,
                                  TopEnt* part_top, int max_blocks, cudaStream_t s,
                                  int* grid_out) {
  SelSrc src;
  memset(&src, 0, sizeof src);
  src.basis = basis;
  src.stride = stride_elems;
  src.id0 = id0;
  src.n = n;
  src.nseg = 1;
  src.nan_notpd = 1;  // the FP64 path marks a nplet that is not positive definite by a NaN
  src.cmb = cmb;
  src.top_m = top_m;
  src.status = status;
  src.ws = ws;
  long long gx = (long long)((n + SEL_PER_BLOCK - 1) / SEL_PER_BLOCK);
  if (gx < 1) gx = 1;
  if (gx > max_blocks - 1) gx = max_blocks - 1;
  if (gx < 1) return cudaErrorInvalidValue;
  return launch_select<double>(src, (int)gx, part, part_top, s, grid_out);
}

cudaError_t launch_select_list64(const double* basis, unsigned long long stride_elems,
                                 const unsigned long long* ids, const unsigned long long* count,
                                 unsigned long long cap, Combine cmb, int top_m,
                                 unsigned char* ws, int* status, PartRec* part, TopEnt* part_top,
                                 int max_blocks, cudaStream_t s, int* grid_out) {
  SelSrc src;
  memset(&src, 0, sizeof src);
  src.basis = basis;
  src.stride = stride_elems;
  src.ids = ids;
  src.counts = count;
  src.n = cap;
  src.nseg = 1;
  src.nan_notpd = 1;
  src.cmb = cmb;
  src.top_m = top_m;
  src.status = status;
  src.ws = ws;
  const int gx = SEL_LIST_BLOCKS < max_blocks - 1 ? SEL_LIST_BLOCKS : max_blocks - 1;
  if (gx < 1) return cudaErrorInvalidValue;
  return launch_select<double>(src, gx, part, part_top, s, grid_out);
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
