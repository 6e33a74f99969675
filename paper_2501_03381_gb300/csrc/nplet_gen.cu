// Generic nplet kernels (any order 1 <= k <= 64): FP64 path, FP64 re-factor of
// the nplets the FP32 path flagged, and the FP32 path for orders above the
// register-resident range.  Also the per-order merge and the device unrank.
#include <type_traits>

#include "nplet_common.cuh"

namespace thoi {

#define IXG(i, j) ((i) * ((i) + 1) / 2 + (j))

// Cholesky of the packed lower triangle A (k x k) in place, then W = L^-1 in
// place column by column, p_j = (R_S^-1)_jj = sum_i W_ij^2.  Returns
// lr = log det R_S (= sum log pivots), sp = sum_j log p_j, the smallest pivot
// and trace(R_S^-1).  `bad` is set for a zero/negative/non-finite product.
template <typename V>
__device__ void chol_loo_gen(V* A, int k, V& lr, V& sp, V& pmin, V& trace, bool& bad) {
  V P1 = 1, P2 = 1;
  int E1 = 0, E2 = 0;
  pmin = pinf<V>();
  for (int p = 0; p < k; p++) {
    const V d = A[IXG(p, p)];
    pmin = d < pmin ? d : pmin;
    bad |= !pivot_ok(d);
    P1 *= d;
    if ((p & 7) == 7 || p == k - 1) renorm(P1, E1, bad);
    const V inv = (V)1 / sqrt(d);
    A[IXG(p, p)] = inv;
    for (int i = p + 1; i < k; i++) A[IXG(i, p)] *= inv;
    for (int i = p + 1; i < k; i++) {
      const V lip = A[IXG(i, p)];
      for (int j = p + 1; j <= i; j++) A[IXG(i, j)] = fma(-lip, A[IXG(j, p)], A[IXG(i, j)]);
    }
  }
  trace = 0;
  for (int j = 0; j < k; j++) {
    const V wjj = A[IXG(j, j)];
    V pj = wjj * wjj;
    for (int i = j + 1; i < k; i++) {
      V s = A[IXG(i, j)] * wjj;
      for (int m = j + 1; m < i; m++) s = fma(A[IXG(i, m)], A[IXG(m, j)], s);
      const V w = -A[IXG(i, i)] * s;
      A[IXG(i, j)] = w;
      pj = fma(w, w, pj);
    }
    trace += pj;
    P2 *= pj;
    if ((j & 7) == 7 || j == k - 1) renorm(P2, E2, bad);
  }
  lr = log_of(P1, E1);
  sp = log_of(P2, E2);
}

template <typename V, typename M>
__device__ __forceinline__ void gather_gen(M mask, int k, int N, const V* sR, int ldr, const V* sls,
                                           V* A, V& lsum) {
  int c[THOI_MAX_N];
  M m = mask;
  for (int i = 0; i < k; i++) {
    const int hb = hibit(m);
    m ^= (M)1 << hb;
    c[i] = N - 1 - hb;
  }
  lsum = 0;
  for (int i = 0; i < k; i++) {
    const V* row = sR + c[i] * ldr;
    lsum += sls[c[i]];
    for (int j = 0; j <= i; j++) A[IXG(i, j)] = row[c[j]];
  }
}

// One nplet in V precision.  In FP32 (FP32_PATH) a nplet is flagged for the
// FP64 re-factor when its smallest pivot is below tau_piv, trace(R_S^-1)
// exceeds tau_tr, or the result is not finite; in FP64 a nplet with a
// non-positive pivot is not positive definite.
template <typename V, int KMAX, bool LIST, bool FP32_PATH, typename M>
__global__ void __launch_bounds__(RED_NT) k_nplet_gen(const NpletArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ RedScratch sc;
  __shared__ int s_tcnt[2];
  __shared__ int s_stop;
  using I = typename std::conditional<LIST, unsigned long long, unsigned>::type;
  const int N = a.N, k = a.k, ldr = row_stride(N);
  const bool red = a.mode == 1;
  const bool with_top = red && a.top_m > 0;
  const SmemLayout L = smem_layout(N, k, ldr, sizeof(V), sizeof(I), with_top);
  if (threadIdx.x == 0) { s_tcnt[0] = s_tcnt[1] = 0; s_stop = 0; }
  load_tables<V>(a, smem, L, FP32_PATH ? (const V*)a.R32 : (const V*)a.R64);
  const unsigned long long* sb = reinterpret_cast<const unsigned long long*>(smem + L.binom);
  const V* sR = reinterpret_cast<const V*>(smem + L.R);
  const V* sls = reinterpret_cast<const V*>(smem + L.ls);
  TopBuf<V, I> tb;
  tb.val[0] = reinterpret_cast<V*>(smem + L.tv0);
  tb.val[1] = reinterpret_cast<V*>(smem + L.tv1);
  tb.idx[0] = reinterpret_cast<I*>(smem + L.ti0);
  tb.idx[1] = reinterpret_cast<I*>(smem + L.ti1);
  tb.cnt = s_tcnt;
  V thr_hi = -pinf<V>(), thr_lo = pinf<V>();
  ThreadRed<V, I> tr;
  tr.init();
  unsigned notpd = 0;
  V A[KMAX * (KMAX + 1) / 2];
  const M full = (N >= (int)(8 * sizeof(M))) ? ~(M)0 : (((M)1 << N) - 1);

  unsigned long long n;
  if (LIST) {
    const unsigned long long c = *a.flag_count;
    n = c < a.flag_cap ? c : a.flag_cap;
  } else {
    n = a.rank_end - a.rank_begin;
  }
  const unsigned long long stride = (unsigned long long)gridDim.x * RED_NT;
  const unsigned long long rounds = (n + stride - 1) / stride;
  const int trigger = TOP_CAP - RED_NT;
  const unsigned long long id_off = LIST ? 0ull : a.id_base + a.rank_begin;
  const CombineV<V> cmbv(a.cmb);

  for (unsigned long long rd = 0; rd < rounds; rd++) {
    const unsigned long long e = rd * stride + (unsigned long long)blockIdx.x * RED_NT + threadIdx.x;
    if (e < n) {
      unsigned long long r, gid;
      if (LIST) {
        gid = a.flag_ids[e];
        r = gid - a.id_base;
      } else {
        r = a.rank_begin + e;
        gid = a.id_base + r;
      }
      const M mask = unrank_s<M>(r, k, N, sb, k + 1);
      V lsum, lr, sp, pmin, trace;
      bool bad = false;
      gather_gen<V, M>(mask, k, N, sR, ldr, sls, A, lsum);
      chol_loo_gen<V>(A, k, lr, sp, pmin, trace, bad);
      V v[5];
      combine5<V>(lr, sp, lsum, cmbv, v);
      if (FP32_PATH) {
        bad |= !(pmin >= (V)a.tau_piv) | !(trace <= (V)a.tau_tr);
      } else if (bad) {
        notpd++;
        atomicOr(a.status, ST_NOT_PD);
#pragma unroll
        for (int m = 0; m < 5; m++) v[m] = pinf<V>() - pinf<V>();  // NaN
      }
      const I loc = LIST ? (I)gid : (I)(r - a.rank_begin);
      if (FP32_PATH && a.mode == 2) {
        store_basis(a, gid, (float)lr, (float)sp, (float)lsum, bad);
      } else if (!red) {
        store5<V>(a, gid, v);
      } else if (!bad) {
        tr.add(v, loc, lr, sp, lsum);
        tr.flush();
        if (with_top) top_offer(tb, v[3], loc, thr_hi, thr_lo);
      }
      if (FP32_PATH) flag_append(a, bad, gid);
    }
    if (threadIdx.x == 0 && a.cancel && *(volatile const int*)a.cancel) s_stop = 1;
    __syncthreads();
    if (with_top) {
      // thresholds move only right after a sort: between sorts the buffer is
      // unordered, and the last sorted M-th entry stays a valid bound
      const bool c0 = tb.cnt[0] > trigger, c1 = tb.cnt[1] > trigger;
      if (c0) {
        top_sort_cut(tb, 0, a.top_m);
        thr_hi = top_threshold(tb, 0, a.top_m);
      }
      if (c1) {
        top_sort_cut(tb, 1, a.top_m);
        thr_lo = top_threshold(tb, 1, a.top_m);
      }
      __syncthreads();
    }
    if (s_stop) {
      if (threadIdx.x == 0) atomicOr(a.status, ST_CANCELLED);
      break;
    }
  }
  if (red) {
    int th = 0, tl = 0;
    if (with_top) {
      top_sort_cut(tb, 0, a.top_m);
      top_sort_cut(tb, 1, a.top_m);
      th = tb.cnt[0];
      tl = tb.cnt[1];
      top_write(tb, a.top_m, id_off, a.part_top + (size_t)blockIdx.x * 2 * a.top_m);
    }
    block_write_part<V, I>(tr, notpd, id_off, sc, a.part + blockIdx.x, th, tl);
  }
}

// ---------------------------------------------------------------- fused records: sample bounds
// Bounds of one order slot's extremes from a sample of its nplets (see the
// fused-records notes in nplet_common.cuh).  Sample i of S = min(n, grid *
// FS_NT * FS_PER) is the nplet of rank rank_begin + floor(i n / S); block b
// takes samples b, b + grid, b + 2 grid, ..., so every block spreads over the
// whole range.  Each sample is evaluated in FP32 by the generic routine; a
// sample the FP32 path would flag is skipped.  Block minima and maxima go
// into the slot's keys with atomicMax (complemented keys where the slot wants
// a minimum): the measures' global minima and maxima, and for the ranked
// measure the largest block minimum and the smallest block maximum.
constexpr int FS_NT = 128;
constexpr int FS_PER = 8;

template <int KMAX, typename M>
__global__ void __launch_bounds__(FS_NT) k_fused_sample(const NpletArgs a, unsigned long long S,
                                                        unsigned* __restrict__ keys) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float s_mn[FS_NT / 32][5], s_mx[FS_NT / 32][5];
  __shared__ unsigned s_valid[FS_NT / 32];
  const int N = a.N, k = a.k, ldr = row_stride(N);
  const SmemLayout L = smem_layout(N, k, ldr, sizeof(float), sizeof(unsigned), 0);
  load_tables<float>(a, smem, L, a.R32);
  const unsigned long long* sb = reinterpret_cast<const unsigned long long*>(smem + L.binom);
  const float* sR = reinterpret_cast<const float*>(smem + L.R);
  const float* sls = reinterpret_cast<const float*>(smem + L.ls);
  const unsigned long long n = a.rank_end - a.rank_begin;
  const unsigned long long q = n / S, rem = n % S;
  const CombineV<float> cv(a.cmb);
  float mn[5], mx[5];
#pragma unroll
  for (int m = 0; m < 5; m++) {
    mn[m] = pinf<float>();
    mx[m] = -pinf<float>();
  }
  unsigned valid = 0;
  float A[KMAX * (KMAX + 1) / 2];
  for (int e = 0; e < FS_PER; e++) {
    const unsigned long long i =
        ((unsigned long long)threadIdx.x * FS_PER + e) * gridDim.x + blockIdx.x;
    if (i >= S) continue;
    const unsigned long long r = a.rank_begin + i * q + (i * rem) / S;
    const M mask = unrank_s<M>(r, k, N, sb, k + 1);
    float lsum, lr, sp, pmin, trace;
    bool bad = false;
    gather_gen<float, M>(mask, k, N, sR, ldr, sls, A, lsum);
    chol_loo_gen<float>(A, k, lr, sp, pmin, trace, bad);
    bad |= !(pmin >= a.tau_piv) | !(trace <= a.tau_tr);
    if (bad) continue;
    float v[5];
    combine5<float>(lr, sp, lsum, cv, v);
#pragma unroll
    for (int m = 0; m < 5; m++) {
      mn[m] = fminf(mn[m], v[m]);
      mx[m] = fmaxf(mx[m], v[m]);
    }
    valid++;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int m = 0; m < 5; m++) {
      mn[m] = fminf(mn[m], __shfl_xor_sync(0xffffffffu, mn[m], o));
      mx[m] = fmaxf(mx[m], __shfl_xor_sync(0xffffffffu, mx[m], o));
    }
    valid += __shfl_xor_sync(0xffffffffu, valid, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int m = 0; m < 5; m++) {
      s_mn[w][m] = mn[m];
      s_mx[w][m] = mx[m];
    }
    s_valid[w] = valid;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned nv = 0;
    for (int q2 = 0; q2 < FS_NT / 32; q2++) {
      nv += s_valid[q2];
      for (int m = 0; m < 5; m++) {
        mn[m] = fminf(mn[m], s_mn[q2][m]);
        mx[m] = fmaxf(mx[m], s_mx[q2][m]);
      }
    }
    if (nv > 0) {
      const int top = a.cmb.top;
      for (int m = 0; m < 5; m++) {
        const unsigned klo = fkey32(mn[m]), khi = fkey32(mx[m]);
        atomicMax(&keys[m], fused_slot_negated(m, top) ? ~klo : klo);
        atomicMax(&keys[5 + m], fused_slot_negated(5 + m, top) ? ~khi : khi);
      }
    }
  }
}

// Samples per thread of the sample bounds: about n / 256 samples in all
// (at least 32K, at most 1M), over max(256, top_m) blocks of 128 threads.
int fused_sample_per_thread(unsigned long long n, int top_m) {
  const unsigned long long grid = top_m > 256 ? (unsigned long long)top_m : 256ull;
  unsigned long long S = n / 256;
  if (S < (1ull << 15)) S = 1ull << 15;
  if (S > (1ull << 20)) S = 1ull << 20;
  unsigned long long e = (S + grid * FS_NT - 1) / (grid * FS_NT);
  return (int)(e < 1 ? 1 : (e > 32 ? 32 : e));
}

cudaError_t launch_fused_sample(const NpletArgs& a0, int num_sms, cudaStream_t s) {
  const unsigned long long n = a0.rank_end - a0.rank_begin;
  if (n == 0) return cudaSuccess;
  if (a0.k <= KREG_MAX) {
    // the one-thread register kernel in its sample mode
    NpletArgs a = a0;
    a.mode = 4;
    Shape sh;
    sh.blocks_per_sm = 0;
    sh.chunk = fused_sample_per_thread(n, a.top_m);
    sh.lanes = 1;
    sh.prefix = 0;
    return launch_nplet_f32(a, sh, num_sms, s, nullptr, 1 << 30);
  }
  NpletArgs a = a0;
  a.mode = 0;  // the sample kernel reads no bounds
  const int grid = a.top_m > 256 ? a.top_m : 256;
  const unsigned long long cap = (unsigned long long)grid * FS_NT * FS_PER;
  const unsigned long long S = n < cap ? n : cap;
  const SmemLayout L = smem_layout(a.N, a.k, row_stride(a.N), sizeof(float), sizeof(unsigned), 0);
  void (*fn)(const NpletArgs, unsigned long long, unsigned*);
  const bool wide = a.N > 32;
  if (a.k <= 8) fn = wide ? k_fused_sample<8, unsigned long long> : k_fused_sample<8, unsigned>;
  else if (a.k <= 16) fn = wide ? k_fused_sample<16, unsigned long long> : k_fused_sample<16, unsigned>;
  else if (a.k <= 32) fn = wide ? k_fused_sample<32, unsigned long long> : k_fused_sample<32, unsigned>;
  else return cudaErrorInvalidValue;
  int occ = 0;
  cudaError_t e = occupancy_cached((const void*)fn, FS_NT, L.total, &occ);
  if (e != cudaSuccess) return e;
  fn<<<grid, FS_NT, L.total, s>>>(a, S, const_cast<unsigned*>(a0.thr_keys));
  return cudaGetLastError();
}

// ---------------------------------------------------------------- merge
// One block per order slot: fold the FP32 partials and the FP64 partials (in
// block order), merge the sorted top lists pairwise by (value, id), and
// write the final record and top lists.
constexpr int MERGE_NT = 128;
constexpr int MERGE_SURV_CAP = 4096;  // survivors sorted in shared memory

// Unsigned key with the numeric order of a double (sign-magnitude to offset
// binary), so the merge orders entries with integer compares: on this GPU a
// double compare runs on the narrow FP64 pipe.
__device__ __forceinline__ unsigned long long dkey(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__device__ __forceinline__ bool ent_before(int side, const TopEnt& a, const TopEnt& b) {
  const unsigned long long ka = dkey(a.v), kb = dkey(b.v);
  if (ka != kb) return side == 0 ? (ka > kb) : (ka < kb);
  return a.id < b.id;
}
__device__ __forceinline__ bool ent_same(const TopEnt& a, const TopEnt& b) {
  return dkey(a.v) == dkey(b.v) && a.id == b.id;
}
__device__ __forceinline__ void kpick_min(double& v, unsigned long long& i, double ov,
                                          unsigned long long oi) {
  const unsigned long long k = dkey(v), ko = dkey(ov);
  if (ko < k || (ko == k && oi < i)) { v = ov; i = oi; }
}
__device__ __forceinline__ void kpick_max(double& v, unsigned long long& i, double ov,
                                          unsigned long long oi) {
  const unsigned long long k = dkey(v), ko = dkey(ov);
  if (ko > k || (ko == k && oi < i)) { v = ov; i = oi; }
}

// Merge sorted lists X (nx) and Y (ny), keep the first `keep` into Z.
__device__ void merge_path(int side, const TopEnt* X, int nx, const TopEnt* Y, int ny, TopEnt* Z,
                           int keep) {
  for (int p = threadIdx.x; p < keep; p += MERGE_NT) {
    // find i in [max(0,p-ny), min(p,nx)] with X[i-1] before-or-eq Y[p-i] and Y[p-i-1] before X[i]
    int lo = p - ny > 0 ? p - ny : 0, hi = p < nx ? p : nx;
    while (lo < hi) {
      const int i = (lo + hi) >> 1;
      const int j = p - i;
      // take more from X if X[i] comes before Y[j-1]
      if (ent_before(side, X[i], Y[j - 1])) lo = i + 1;
      else hi = i;
    }
    const int i = lo, j = p - lo;
    TopEnt out;
    if (i < nx && (j >= ny || ent_before(side, X[i], Y[j]))) out = X[i];
    else out = Y[j];
    Z[p] = out;
  }
}

__device__ void merge_slot(const MergeDesc& d, const PartRec* __restrict__ p32base,
                           const TopEnt* __restrict__ t32base, const PartRec* __restrict__ p64base,
                           const TopEnt* __restrict__ t64base, int top_m,
                           thoi_order_record* __restrict__ rec, TopEnt* __restrict__ top_out,
                           unsigned char* smem);

__global__ void __launch_bounds__(MERGE_NT) k_merge(const MergeDescs D,
                                                    const PartRec* __restrict__ p32base,
                                                    const TopEnt* __restrict__ t32base,
                                                    const PartRec* __restrict__ p64base,
                                                    const TopEnt* __restrict__ t64base, int top_m,
                                                    thoi_order_record* __restrict__ recs,
                                                    TopEnt* __restrict__ tops) {
  extern __shared__ __align__(16) unsigned char smem[];
  merge_slot(D.d[blockIdx.x], p32base, t32base, p64base, t64base, top_m, recs + blockIdx.x,
             tops + (size_t)blockIdx.x * 2 * top_m, smem);
}

// Batched form: one block per slot, descriptors and output places in device
// memory (any number of slots).
__global__ void __launch_bounds__(MERGE_NT) k_merge_arr(const MergeDesc* __restrict__ D,
                                                        const PartRec* __restrict__ p32base,
                                                        const TopEnt* __restrict__ t32base,
                                                        const PartRec* __restrict__ p64base,
                                                        const TopEnt* __restrict__ t64base,
                                                        int top_m,
                                                        thoi_order_record* const* __restrict__ recp,
                                                        TopEnt* const* __restrict__ topp) {
  extern __shared__ __align__(16) unsigned char smem[];
  merge_slot(D[blockIdx.x], p32base, t32base, p64base, t64base, top_m, recp[blockIdx.x],
             topp[blockIdx.x], smem);
}

__device__ void merge_slot(const MergeDesc& d, const PartRec* __restrict__ p32base,
                           const TopEnt* __restrict__ t32base, const PartRec* __restrict__ p64base,
                           const TopEnt* __restrict__ t64base, int top_m,
                           thoi_order_record* __restrict__ rec, TopEnt* __restrict__ top_out,
                           unsigned char* smem) {
  const PartRec* p32 = p32base + d.p32_off;
  const TopEnt* t32 = t32base + (size_t)d.p32_off * 2 * top_m;
  const PartRec* p64 = p64base + d.p64_off;
  const TopEnt* t64 = t64base + (size_t)d.p64_off * 2 * top_m;
  const int g32 = d.g32, g64 = d.g64, k = d.k;
  const Combine cmb = d.cmb;
  const unsigned long long* refactored = d.refactored;
  __shared__ double s_vmin[MERGE_NT][5];
  __shared__ unsigned long long s_imin[MERGE_NT][5];
  __shared__ double s_vmax[MERGE_NT][5];
  __shared__ unsigned long long s_imax[MERGE_NT][5];
  __shared__ double s_sum[MERGE_NT][3];
  __shared__ unsigned long long s_cnt[MERGE_NT][3];
  const int G = g32 + g64;
  // 1) scalar fields: each thread folds partials t, t+NT, ... in order.
  double vmn[5], vmx[5], sum[3] = {0, 0, 0};
  unsigned long long imn[5], imx[5], cnt = 0, neg = 0, npd = 0;
  for (int m = 0; m < 5; m++) {
    vmn[m] = pinf<double>();
    vmx[m] = -pinf<double>();
    imn[m] = imx[m] = ~0ull;
  }
  for (int b = threadIdx.x; b < G; b += MERGE_NT) {
    const PartRec& P = b < g32 ? p32[b] : p64[b - g32];
    npd += P.notpd;
    // a partial without nplets holds +-inf extremes with id ~0, which never
    // win; the candidate partials of fused records carry extremes only
    for (int m = 0; m < 5; m++) {
      kpick_min(vmn[m], imn[m], P.vmin[m], P.imin[m]);
      kpick_max(vmx[m], imx[m], P.vmax[m], P.imax[m]);
    }
    sum[0] += P.s_lr;
    sum[1] += P.s_sp;
    sum[2] += P.s_ls;
    cnt += P.count;
    neg += P.neg;
  }
  for (int m = 0; m < 5; m++) {
    s_vmin[threadIdx.x][m] = vmn[m];
    s_imin[threadIdx.x][m] = imn[m];
    s_vmax[threadIdx.x][m] = vmx[m];
    s_imax[threadIdx.x][m] = imx[m];
  }
  s_sum[threadIdx.x][0] = sum[0];
  s_sum[threadIdx.x][1] = sum[1];
  s_sum[threadIdx.x][2] = sum[2];
  s_cnt[threadIdx.x][0] = cnt;
  s_cnt[threadIdx.x][1] = neg;
  s_cnt[threadIdx.x][2] = npd;
  __syncthreads();
  for (int h = MERGE_NT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      const int o = threadIdx.x + h;
      for (int m = 0; m < 5; m++) {
        kpick_min(s_vmin[threadIdx.x][m], s_imin[threadIdx.x][m], s_vmin[o][m], s_imin[o][m]);
        kpick_max(s_vmax[threadIdx.x][m], s_imax[threadIdx.x][m], s_vmax[o][m], s_imax[o][m]);
      }
      for (int q = 0; q < 3; q++) {
        s_sum[threadIdx.x][q] += s_sum[o][q];
        s_cnt[threadIdx.x][q] += s_cnt[o][q];
      }
    }
    __syncthreads();
  }
  const unsigned long long total = s_cnt[0][0];
  if (threadIdx.x == 0) {
    thoi_order_record R;
    R.k = k;
    R.count = total + s_cnt[0][2];
    R.count_neg_O = s_cnt[0][1];
    R.n_refactored = refactored ? *refactored : 0ull;
    R.n_not_pd = s_cnt[0][2];
    R.top_count = (int)(total < (unsigned long long)top_m ? total : (unsigned long long)top_m);
    const double inv = total ? 1.0 / (double)total : 0.0;
    const double mlr = s_sum[0][0] * inv, msp = s_sum[0][1] * inv, mls = s_sum[0][2] * inv;
    const double tc = -0.5 * mlr + cmb.tc_c, dtc = 0.5 * (mlr + msp) + cmb.dtc_c;
    R.mean[0] = cmb.h_c + 0.5 * (mlr + mls);
    R.mean[1] = tc;
    R.mean[2] = dtc;
    R.mean[3] = tc - dtc;
    R.mean[4] = tc + dtc;
    for (int m = 0; m < 5; m++) {
      R.min[m] = total ? s_vmin[0][m] : 0.0;
      R.max[m] = total ? s_vmax[0][m] : 0.0;
      R.argmin[m] = total ? s_imin[0][m] : ~0ull;
      R.argmax[m] = total ? s_imax[0][m] : ~0ull;
      if (!total) R.mean[m] = 0.0;
    }
    *rec = R;
    if (d.thr_keys && total) {
      // fused records: every extreme must lie within its bound, so that no
      // nplet left off the candidate list could have replaced it
      bool ok = true;
      for (int m = 0; m < 5; m++) {
        ok &= R.min[m] <= (double)fused_threshold(d.thr_keys[m], m, cmb.top);
        ok &= R.max[m] >= (double)fused_threshold(d.thr_keys[5 + m], 5 + m, cmb.top);
      }
      if (!ok) atomicOr(d.status, ST_INEXACT);
    }
  }
  // 2) top lists
  if (top_m <= 0) return;
  TopEnt* bufA = reinterpret_cast<TopEnt*>(smem);
  TopEnt* bufB = bufA + top_m;
  TopEnt* stage = bufB + top_m;
  TopEnt* surv = stage + top_m;                              // MERGE_SURV_CAP entries
  int* offs = reinterpret_cast<int*>(surv + MERGE_SURV_CAP);  // G + 1 entries
  __shared__ TopEnt s_best[MERGE_NT];
  __shared__ int s_have[MERGE_NT];
  __shared__ int s_total;
  for (int side = 0; side < 2; side++) {
    // (a) threshold: the best M-th entry among the blocks with a full list.
    // Such a block alone holds M entries at least that good, so the global
    // top M is among the entries of all lists that are at least that good.
    {
      TopEnt best;
      best.v = 0.0;
      best.id = ~0ull;
      int have = 0;
      for (int b = threadIdx.x; b < G; b += MERGE_NT) {
        const PartRec& P = b < g32 ? p32[b] : p64[b - g32];
        const int nl = side == 0 ? P.top_hi : P.top_lo;
        if (nl < top_m) continue;
        const TopEnt* Lst = (b < g32 ? t32 + (size_t)b * 2 * top_m
                                     : t64 + (size_t)(b - g32) * 2 * top_m) + (size_t)side * top_m;
        const TopEnt e = Lst[top_m - 1];
        if (!have || ent_before(side, e, best)) { best = e; have = 1; }
      }
      s_best[threadIdx.x] = best;
      s_have[threadIdx.x] = have;
      __syncthreads();
      for (int h = MERGE_NT / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
          const int o = threadIdx.x + h;
          if (s_have[o] && (!s_have[threadIdx.x] || ent_before(side, s_best[o], s_best[threadIdx.x]))) {
            s_best[threadIdx.x] = s_best[o];
            s_have[threadIdx.x] = 1;
          }
        }
        __syncthreads();
      }
    }
    const bool have = s_have[0] != 0;
    const TopEnt thr = s_best[0];
    bool done = false;
    if (have) {
      // (b) survivors per list (binary search for the entries at least as good)
      for (int b = threadIdx.x; b < G; b += MERGE_NT) {
        const PartRec& P = b < g32 ? p32[b] : p64[b - g32];
        const int nl = side == 0 ? P.top_hi : P.top_lo;
        const TopEnt* Lst = (b < g32 ? t32 + (size_t)b * 2 * top_m
                                     : t64 + (size_t)(b - g32) * 2 * top_m) + (size_t)side * top_m;
        int lo = 0, hi = nl > 0 ? nl : 0;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          const TopEnt e = Lst[mid];
          const bool keep = ent_before(side, e, thr) || ent_same(e, thr);
          if (keep) lo = mid + 1;
          else hi = mid;
        }
        offs[b + 1] = lo;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        offs[0] = 0;
        for (int b = 0; b < G; b++) offs[b + 1] += offs[b];
        s_total = offs[G];
      }
      __syncthreads();
      const int S = s_total;
      if (S <= MERGE_SURV_CAP) {
        // (c) gather the survivors, sort them (bitonic), keep the first M
        for (int q = threadIdx.x; q < S; q += MERGE_NT) {
          int lo = 0, hi = G - 1;  // list b with offs[b] <= q < offs[b + 1]
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (offs[mid] <= q) lo = mid;
            else hi = mid - 1;
          }
          const int b = lo;
          const TopEnt* Lst = (b < g32 ? t32 + (size_t)b * 2 * top_m
                                       : t64 + (size_t)(b - g32) * 2 * top_m) + (size_t)side * top_m;
          surv[q] = Lst[q - offs[b]];
        }
        int P2 = 2;
        while (P2 < S) P2 <<= 1;
        for (int q = S + threadIdx.x; q < P2; q += MERGE_NT) {
          surv[q].v = side == 0 ? -pinf<double>() : pinf<double>();
          surv[q].id = ~0ull;
        }
        __syncthreads();
        for (int kk = 2; kk <= P2; kk <<= 1) {
          for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P2; i += MERGE_NT) {
              const int ixj = i ^ j;
              if (ixj > i) {
                const bool up = (i & kk) == 0;
                const TopEnt x = surv[i], y = surv[ixj];
                const bool sw = up ? ent_before(side, y, x) : ent_before(side, x, y);
                if (sw) { surv[i] = y; surv[ixj] = x; }
              }
            }
            __syncthreads();
          }
        }
        const int nout = S < top_m ? S : top_m;
        for (int q = threadIdx.x; q < top_m; q += MERGE_NT) {
          TopEnt e;
          if (q < nout) e = surv[q];
          else { e.v = 0.0; e.id = ~0ull; }
          top_out[(size_t)side * top_m + q] = e;
        }
        __syncthreads();
        done = true;
      }
    }
    if (done) continue;
    // fallback: pairwise merge of the sorted lists
    int ncur = 0;
    TopEnt* cur = bufA;
    TopEnt* nxt = bufB;
    for (int b = 0; b < G; b++) {
      const PartRec& P = b < g32 ? p32[b] : p64[b - g32];
      const int nl = side == 0 ? P.top_hi : P.top_lo;
      if (nl <= 0) continue;
      const TopEnt* Lst = (b < g32 ? t32 + (size_t)b * 2 * top_m : t64 + (size_t)(b - g32) * 2 * top_m) +
                          (size_t)side * top_m;
      // a full current list that the block's best entry cannot enter: skip
      if (ncur == top_m && !ent_before(side, Lst[0], cur[top_m - 1])) continue;
      for (int q = threadIdx.x; q < nl; q += MERGE_NT) stage[q] = Lst[q];
      __syncthreads();
      const int keep = ncur + nl < top_m ? ncur + nl : top_m;
      merge_path(side, cur, ncur, stage, nl, nxt, keep);
      __syncthreads();
      TopEnt* t = cur; cur = nxt; nxt = t;
      ncur = keep;
    }
    for (int q = threadIdx.x; q < top_m; q += MERGE_NT) {
      TopEnt e;
      if (q < ncur) e = cur[q];
      else { e.v = 0.0; e.id = ~0ull; }
      top_out[(size_t)side * top_m + q] = e;
    }
    __syncthreads();
  }
  if (d.thr_keys && threadIdx.x == 0) {
    // fused records: a list must hold min(count, M) entries, and a list of
    // M entries must end beyond its bound (every nplet off the candidate list
    // lies strictly inside the bound, so it could not have entered)
    const unsigned long long want = total < (unsigned long long)top_m ? total : top_m;
    bool ok = true;
    for (int side = 0; side < 2; side++) {
      const TopEnt* Lst = top_out + (size_t)side * top_m;
      unsigned long long have = 0;
      for (int q = 0; q < top_m; q++) have += Lst[q].id != ~0ull ? 1ull : 0ull;
      ok &= have >= want;
      if (total > (unsigned long long)top_m && have >= (unsigned long long)top_m) {
        const int j = side == 0 ? 5 + cmb.top : cmb.top;
        const double t = (double)fused_threshold(d.thr_keys[j], j, cmb.top);
        ok &= side == 0 ? Lst[top_m - 1].v >= t : Lst[top_m - 1].v <= t;
      }
    }
    if (!ok) atomicOr(d.status, ST_INEXACT);
  }
}

// ---------------------------------------------------------------- device unrank (test hook)
__global__ void k_unrank_ids(int N, const int* __restrict__ orders,
                             const unsigned long long* __restrict__ offsets, int n_orders,
                             const unsigned long long* __restrict__ binom,
                             const unsigned long long* __restrict__ ids, long long n, int kmax,
                             int8_t* __restrict__ out) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const unsigned long long id = ids[q];
  int s = 0;
  while (s + 1 < n_orders && id >= offsets[s + 1]) s++;
  int8_t* row = out + (size_t)q * kmax;
  if (id >= offsets[n_orders]) {
    for (int i = 0; i < kmax; i++) row[i] = -2;
    return;
  }
  const int k = orders[s];
  const unsigned long long mask = unrank_mask<unsigned long long>(id - offsets[s], k, N, binom);
  unsigned long long m = mask;
  for (int i = 0; i < kmax; i++) {
    if (i < k) {
      const int hb = hibit(m);
      m ^= 1ull << hb;
      row[i] = (int8_t)(N - 1 - hb);
    } else {
      row[i] = -1;
    }
  }
}

// ---------------------------------------------------------------- launchers
template <typename V, int KMAX, bool LIST, bool FP32_PATH>
static cudaError_t launch_gen_t(const NpletArgs& a, int num_sms, cudaStream_t s, int* grid_out,
                                int max_blocks) {
  const bool red = a.mode == 1;
  using I = typename std::conditional<LIST, unsigned long long, unsigned>::type;
  const SmemLayout L = smem_layout(a.N, a.k, row_stride(a.N), sizeof(V), sizeof(I),
                                   red && a.top_m > 0);
  const bool wide = a.N > 32;
  cudaError_t e;
  void (*fn)(const NpletArgs);
  if (wide) fn = k_nplet_gen<V, KMAX, LIST, FP32_PATH, unsigned long long>;
  else fn = k_nplet_gen<V, KMAX, LIST, FP32_PATH, unsigned>;
  int occ = 0;
  e = occupancy_cached((const void*)fn, RED_NT, L.total, &occ);
  if (e != cudaSuccess) return e;
  long long grid = (long long)num_sms * occ;
  if (!LIST) {
    const unsigned long long n = a.rank_end - a.rank_begin;
    const long long need = (long long)((n + RED_NT - 1) / RED_NT);
    if (need < grid) grid = need > 0 ? need : 1;
  }
  if (grid > max_blocks) grid = max_blocks;
  fn<<<(unsigned)grid, RED_NT, L.total, s>>>(a);
  if (grid_out) *grid_out = (int)grid;
  return cudaGetLastError();
}

int gen_kmax_bucket(int k) { return k <= 8 ? 8 : (k <= 16 ? 16 : (k <= 32 ? 32 : 64)); }

cudaError_t launch_nplet_f64(const NpletArgs& a, int num_sms, cudaStream_t s, int* grid_out,
                             int max_blocks) {
  switch (gen_kmax_bucket(a.k)) {
    case 8: return launch_gen_t<double, 8, false, false>(a, num_sms, s, grid_out, max_blocks);
    case 16: return launch_gen_t<double, 16, false, false>(a, num_sms, s, grid_out, max_blocks);
    case 32: return launch_gen_t<double, 32, false, false>(a, num_sms, s, grid_out, max_blocks);
    default: return launch_gen_t<double, 64, false, false>(a, num_sms, s, grid_out, max_blocks);
  }
}

cudaError_t launch_refactor(const NpletArgs& a, int num_sms, cudaStream_t s, int* grid_out,
                            int max_blocks) {
  switch (gen_kmax_bucket(a.k)) {
    case 8: return launch_gen_t<double, 8, true, false>(a, num_sms, s, grid_out, max_blocks);
    case 16: return launch_gen_t<double, 16, true, false>(a, num_sms, s, grid_out, max_blocks);
    case 32: return launch_gen_t<double, 32, true, false>(a, num_sms, s, grid_out, max_blocks);
    default: return launch_gen_t<double, 64, true, false>(a, num_sms, s, grid_out, max_blocks);
  }
}

cudaError_t launch_nplet_f32_gen(const NpletArgs& a, int num_sms, cudaStream_t s, int* grid_out,
                                 int max_blocks) {
  switch (gen_kmax_bucket(a.k)) {
    case 8: return launch_gen_t<float, 8, false, true>(a, num_sms, s, grid_out, max_blocks);
    case 16: return launch_gen_t<float, 16, false, true>(a, num_sms, s, grid_out, max_blocks);
    case 32: return launch_gen_t<float, 32, false, true>(a, num_sms, s, grid_out, max_blocks);
    default: return launch_gen_t<float, 64, false, true>(a, num_sms, s, grid_out, max_blocks);
  }
}

cudaError_t launch_merge(const MergeDescs& D, int n_slots, const PartRec* p32, const TopEnt* t32,
                         const PartRec* p64, const TopEnt* t64, int top_m, thoi_order_record* recs,
                         TopEnt* tops, cudaStream_t s) {
  int gmax = 0;
  for (int i = 0; i < n_slots; i++) gmax = D.d[i].g32 + D.d[i].g64 > gmax ? D.d[i].g32 + D.d[i].g64 : gmax;
  const size_t sm = top_m > 0 ? (size_t)3 * top_m * sizeof(TopEnt) + MERGE_SURV_CAP * sizeof(TopEnt) +
                                    (size_t)(gmax + 1) * sizeof(int)
                              : 0;
  cudaError_t e = cudaFuncSetAttribute(k_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  if (n_slots <= 0) return cudaSuccess;
  k_merge<<<n_slots, MERGE_NT, sm, s>>>(D, p32, t32, p64, t64, top_m, recs, tops);
  return cudaGetLastError();
}

cudaError_t launch_merge_arr(const MergeDesc* D, int n_slots, int gmax, const PartRec* p32,
                             const TopEnt* t32, const PartRec* p64, const TopEnt* t64, int top_m,
                             thoi_order_record* const* recp, TopEnt* const* topp,
                             cudaStream_t s) {
  const size_t sm = top_m > 0 ? (size_t)3 * top_m * sizeof(TopEnt) + MERGE_SURV_CAP * sizeof(TopEnt) +
                                    (size_t)(gmax + 1) * sizeof(int)
                              : 0;
  int occ = 0;
  cudaError_t e = occupancy_cached((const void*)k_merge_arr, MERGE_NT, sm, &occ);
  if (e != cudaSuccess) return e;
  if (n_slots <= 0) return cudaSuccess;
  k_merge_arr<<<n_slots, MERGE_NT, sm, s>>>(D, p32, t32, p64, t64, top_m, recp, topp);
  return cudaGetLastError();
}

cudaError_t launch_unrank_ids(int N, const int* d_orders, const unsigned long long* d_offsets,
                              int n_orders, const unsigned long long* binom,
                              const unsigned long long* ids, long long n, int kmax,
                              int8_t* idx_out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_unrank_ids<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(N, d_orders, d_offsets, n_orders, binom,
                                                           ids, n, kmax, idx_out);
  return cudaGetLastError();
}

}  // namespace thoi
