// Device building blocks of the nplet kernels: per-thread and per-block
// reduction state, the top-M candidate buffers, shared-memory layout, and the
// combine step.  Included by the nplet translation units only.
#pragma once

#include <float.h>

#include "internal.cuh"

namespace thoi {

constexpr double LN2 = 0.69314718055994530942;

template <typename T>
__device__ __forceinline__ T pinf();
template <>
__device__ __forceinline__ float pinf<float>() { return __int_as_float(0x7f800000); }
template <>
__device__ __forceinline__ double pinf<double>() { return __longlong_as_double(0x7ff0000000000000ll); }

template <typename I>
__device__ __forceinline__ I imax_val();
template <>
__device__ __forceinline__ unsigned imax_val<unsigned>() { return 0xffffffffu; }
template <>
__device__ __forceinline__ unsigned long long imax_val<unsigned long long>() { return ~0ull; }

// Binomial lookup in a shared-memory table of stride bs (C(n, m), m < bs).
__device__ __forceinline__ unsigned long long binom_s(const unsigned long long* b, int bs, int n,
                                                      int m) {
  return b[n * bs + m];
}

// Combinatorial-number-system unrank (see unrank_mask) on a table of stride bs.
template <typename M>
__device__ __forceinline__ M unrank_s(unsigned long long r, int k, int N,
                                      const unsigned long long* b, int bs) {
  unsigned long long rr = binom_s(b, bs, N, k) - 1ull - r;
  M mask = 0;
  int d = N - 1;
  for (int i = 0; i < k; i++) {
    const int m = k - i;
    unsigned long long cd = binom_s(b, bs, d, m);
    while (cd > rr) {
      d--;
      cd = binom_s(b, bs, d, m);
    }
    rr -= cd;
    mask |= (M)1 << d;
    d--;
  }
  return mask;
}

// Keep a running product in [1, 2) and its binary exponent apart, so the
// product of up to 64 pivots or inverse diagonals cannot overflow or
// underflow.  `bad` records a zero, denormal, Inf or NaN product.
__device__ __forceinline__ void renorm(float& P, int& E, bool& bad) {
  const int b = __float_as_int(P);
  const int ex = (b >> 23) & 0xff;
  bad |= (ex == 0) | (ex == 255) | (b < 0);
  E += ex - 127;
  P = __int_as_float((b & 0x007fffff) | 0x3f800000);
}
__device__ __forceinline__ void renorm(double& P, int& E, bool& bad) {
  const long long b = __double_as_longlong(P);
  const int ex = (int)((b >> 52) & 0x7ff);
  bad |= (ex == 0) | (ex == 0x7ff) | (b < 0);
  E += ex - 1023;
  P = __longlong_as_double((b & 0x000fffffffffffffll) | 0x3ff0000000000000ll);
}
// NaN test in the value's own precision.  (The library isnan may promote a
// float to double, and a float-to-double conversion runs on the narrow FP64
// pipe of this GPU: one per element bounded the streaming reduction.)
template <typename V>
__device__ __forceinline__ bool is_nan(V x) { return x != x; }

// Reciprocal by the hardware approximation (about 1 ulp), one instruction.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float log_of(float P, int E) {
  return (__log2f(P) + (float)E) * (float)LN2;
}
__device__ __forceinline__ double log_of(double P, int E) { return log(P) + (double)E * LN2; }

// The five measures from the three per-nplet quantities (Methods eqs. TC,
// DTC, O-info, S-info with H from Supp. eq. gaussian_differential_entropy):
// Lr = log det R_S, Sp = sum_j log (R_S^-1)_jj, Ls = sum_{i in S} log Sigma_ii.
// Unsigned key with the numeric order of a double (zeros of both signs map to
// one key).  Double compares run on the narrow FP64 pipe of this GPU; the
// reductions and sorts order doubles through these integer keys instead.
__device__ __forceinline__ unsigned long long okey(double v) {
  unsigned long long u = (unsigned long long)__double_as_longlong(v);
  if ((u << 1) == 0) u = 0;
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// The combine constants in the working precision, converted once per kernel
// (a double-to-float conversion runs on the FP64 pipe).
template <typename V>
struct CombineV {
  V h_c, tc_c, dtc_c;
  __device__ __forceinline__ explicit CombineV(const Combine& c)
      : h_c((V)c.h_c), tc_c((V)c.tc_c), dtc_c((V)c.dtc_c) {}
};

// One of the five combined values by runtime index (selects, no local memory).
template <typename V>
__device__ __forceinline__ V pick5(const V (&v)[5], int m) {
  V r = v[3];
  r = m == 0 ? v[0] : r;
  r = m == 1 ? v[1] : r;
  r = m == 2 ? v[2] : r;
  r = m == 4 ? v[4] : r;
  return r;
}

template <typename V>
__device__ __forceinline__ void combine5(V lr, V sp, V lsum, const CombineV<V>& c, V (&v)[5]) {
  const V tc = (V)(-0.5) * lr + c.tc_c;
  const V dtc = (V)0.5 * (lr + sp) + c.dtc_c;
  v[0] = c.h_c + (V)0.5 * (lr + lsum);
  v[1] = tc;
  v[2] = dtc;
  v[3] = tc - dtc;
  v[4] = tc + dtc;
}

// ---------------------------------------------------------------- reduction state
// Ordering used everywhere: for min, (value, id) ascending; for max, value
// descending then id ascending.  So ties go to the smallest id.
template <typename V, typename I>
struct ThreadRed {
  V mn[5], mx[5];
  I imn[5], imx[5];
  // Running sums in the working precision; in FP32 with Kahan compensation
  // (c*), so that no double arithmetic runs per element: on this GPU the FP64
  // pipe is narrow enough that even one double add per few elements bounds a
  // streaming kernel.
  V plr, psp, pls;
  V clr, csp, cls;
  unsigned cnt, neg;

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int m = 0; m < 5; m++) {
      mn[m] = pinf<V>();
      mx[m] = -pinf<V>();
      imn[m] = imax_val<I>();
      imx[m] = imax_val<I>();
    }
    plr = psp = pls = (V)0;
    clr = csp = cls = (V)0;
    cnt = neg = 0;
  }
  // (kept for the call sites; the compensated sums need no periodic flush)
  __device__ __forceinline__ void flush() {}
  __device__ __forceinline__ static void kahan(V& s, V& c, V x) {
    if (sizeof(V) == 4) {
      const V y = x - c;
      const V t = s + y;
      c = (t - s) - y;
      s = t;
    } else {
      s += x;
    }
  }
  __device__ __forceinline__ double total_lr() const { return (double)plr - (double)clr; }
  __device__ __forceinline__ double total_sp() const { return (double)psp - (double)csp; }
  __device__ __forceinline__ double total_ls() const { return (double)pls - (double)cls; }
  // ids in any order: ties go to the smaller id (branch-free selects; doubles
  // are compared through their integer keys)
  __device__ __forceinline__ void add(const V (&v)[5], I id, V lr, V sp, V lsum) {
    if (sizeof(V) == 8) {
#pragma unroll
      for (int m = 0; m < 5; m++) {
        const unsigned long long kv = okey((double)v[m]), kn = okey((double)mn[m]),
                                 kx = okey((double)mx[m]);
        const bool lt = (kv < kn) | ((kv == kn) & (id < imn[m]));
        const bool gt = (kv > kx) | ((kv == kx) & (id < imx[m]));
        mn[m] = lt ? v[m] : mn[m];
        imn[m] = lt ? id : imn[m];
        mx[m] = gt ? v[m] : mx[m];
        imx[m] = gt ? id : imx[m];
      }
      accumulate(v, lr, sp, lsum);
      return;
    }
#pragma unroll
    for (int m = 0; m < 5; m++) {
      const bool lt = (v[m] < mn[m]) | ((v[m] == mn[m]) & (id < imn[m]));
      const bool gt = (v[m] > mx[m]) | ((v[m] == mx[m]) & (id < imx[m]));
      mn[m] = lt ? v[m] : mn[m];
      imn[m] = lt ? id : imn[m];
      mx[m] = gt ? v[m] : mx[m];
      imx[m] = gt ? id : imx[m];
    }
    accumulate(v, lr, sp, lsum);
  }
  // ids strictly increasing in this thread: a later equal value never wins
  __device__ __forceinline__ void add_mono(const V (&v)[5], I id, V lr, V sp, V lsum) {
#pragma unroll
    for (int m = 0; m < 5; m++) {
      const bool lt = v[m] < mn[m];
      const bool gt = v[m] > mx[m];
      mn[m] = lt ? v[m] : mn[m];
      imn[m] = lt ? id : imn[m];
      mx[m] = gt ? v[m] : mx[m];
      imx[m] = gt ? id : imx[m];
    }
    accumulate(v, lr, sp, lsum);
  }
  __device__ __forceinline__ void accumulate(const V (&v)[5], V lr, V sp, V lsum) {
    kahan(plr, clr, lr);
    kahan(psp, csp, sp);
    kahan(pls, cls, lsum);
    cnt++;
    neg += (v[3] < (V)0) ? 1u : 0u;
  }
};

template <typename V, typename I>
__device__ __forceinline__ void pick_min(V& v, I& i, V ov, I oi) {
  if (ov < v || (ov == v && oi < i)) { v = ov; i = oi; }
}
template <typename V, typename I>
__device__ __forceinline__ void pick_max(V& v, I& i, V ov, I oi) {
  if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
}
template <typename I>
__device__ __forceinline__ void pick_min(double& v, I& i, double ov, I oi) {
  const unsigned long long k = okey(v), ko = okey(ov);
  if (ko < k || (ko == k && oi < i)) { v = ov; i = oi; }
}
template <typename I>
__device__ __forceinline__ void pick_max(double& v, I& i, double ov, I oi) {
  const unsigned long long k = okey(v), ko = okey(ov);
  if (ko > k || (ko == k && oi < i)) { v = ov; i = oi; }
}

struct RedScratch {
  double vmin[RED_NT / 32][5], vmax[RED_NT / 32][5];
  unsigned long long imin[RED_NT / 32][5], imax[RED_NT / 32][5];
  double slr[RED_NT / 32], ssp[RED_NT / 32], sls[RED_NT / 32];
  unsigned long long cnt[RED_NT / 32], neg[RED_NT / 32], notpd[RED_NT / 32];
};

// Block reduction (fixed butterfly then fixed warp order) into one PartRec.
// id_off converts a thread's index type to a global id.
template <typename V, typename I>
__device__ void block_write_part(ThreadRed<V, I>& t, unsigned notpd, unsigned long long id_off,
                                 RedScratch& sc, PartRec* out, int top_hi, int top_lo) {
  t.flush();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long gmn[5], gmx[5];
  double vmn[5], vmx[5];
#pragma unroll
  for (int m = 0; m < 5; m++) {
    vmn[m] = (double)t.mn[m];
    vmx[m] = (double)t.mx[m];
    gmn[m] = (t.imn[m] == imax_val<I>()) ? ~0ull : (unsigned long long)t.imn[m] + id_off;
    gmx[m] = (t.imx[m] == imax_val<I>()) ? ~0ull : (unsigned long long)t.imx[m] + id_off;
  }
  double slr = t.total_lr(), ssp = t.total_sp(), sls = t.total_ls();
  unsigned long long cnt = t.cnt, neg = t.neg, npd = notpd;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int m = 0; m < 5; m++) {
      pick_min(vmn[m], gmn[m], __shfl_xor_sync(0xffffffffu, vmn[m], o),
               __shfl_xor_sync(0xffffffffu, gmn[m], o));
      pick_max(vmx[m], gmx[m], __shfl_xor_sync(0xffffffffu, vmx[m], o),
               __shfl_xor_sync(0xffffffffu, gmx[m], o));
    }
    slr += __shfl_xor_sync(0xffffffffu, slr, o);
    ssp += __shfl_xor_sync(0xffffffffu, ssp, o);
    sls += __shfl_xor_sync(0xffffffffu, sls, o);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    neg += __shfl_xor_sync(0xffffffffu, neg, o);
    npd += __shfl_xor_sync(0xffffffffu, npd, o);
  }
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < 5; m++) {
      sc.vmin[w][m] = vmn[m];
      sc.vmax[w][m] = vmx[m];
      sc.imin[w][m] = gmn[m];
      sc.imax[w][m] = gmx[m];
    }
    sc.slr[w] = slr;
    sc.ssp[w] = ssp;
    sc.sls[w] = sls;
    sc.cnt[w] = cnt;
    sc.neg[w] = neg;
    sc.notpd[w] = npd;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    PartRec r;
    for (int m = 0; m < 5; m++) {
      r.vmin[m] = sc.vmin[0][m];
      r.imin[m] = sc.imin[0][m];
      r.vmax[m] = sc.vmax[0][m];
      r.imax[m] = sc.imax[0][m];
    }
    r.s_lr = sc.slr[0];
    r.s_sp = sc.ssp[0];
    r.s_ls = sc.sls[0];
    r.count = sc.cnt[0];
    r.neg = sc.neg[0];
    r.notpd = sc.notpd[0];
    for (int q = 1; q < RED_NT / 32; q++) {
      for (int m = 0; m < 5; m++) {
        pick_min(r.vmin[m], r.imin[m], sc.vmin[q][m], sc.imin[q][m]);
        pick_max(r.vmax[m], r.imax[m], sc.vmax[q][m], sc.imax[q][m]);
      }
      r.s_lr += sc.slr[q];
      r.s_sp += sc.ssp[q];
      r.s_ls += sc.sls[q];
      r.count += sc.cnt[q];
      r.neg += sc.neg[q];
      r.notpd += sc.notpd[q];
    }
    r.top_hi = top_hi;
    r.top_lo = top_lo;
    *out = r;
  }
}

// ---------------------------------------------------------------- top-M buffers
// Two candidate buffers in shared memory (side 0: largest O, side 1:
// smallest O).  A nplet is appended when it is at least as good as the
// current M-th entry; when a buffer could overflow in the next round, it is
// sorted (bitonic, by (value, id)) and cut back to M entries.
template <typename V, typename I>
struct TopBuf {
  V* val[2];
  I* idx[2];
  int* cnt;  // [2], shared
};

template <typename V, typename I>
__device__ __forceinline__ bool top_before(int side, V va, I ia, V vb, I ib) {
  if (va != vb) return side == 0 ? (va > vb) : (va < vb);
  return ia < ib;
}
template <typename I>
__device__ __forceinline__ bool top_before(int side, double va, I ia, double vb, I ib) {
  const unsigned long long ka = okey(va), kb = okey(vb);
  if (ka != kb) return side == 0 ? (ka > kb) : (ka < kb);
  return ia < ib;
}

template <typename V, typename I>
__device__ void top_sort_cut(TopBuf<V, I>& tb, int side, int M) {
  __syncthreads();
  const int c = tb.cnt[side];
  int P = 2;
  while (P < c) P <<= 1;
  V* val = tb.val[side];
  I* idx = tb.idx[side];
  const V sent = side == 0 ? -pinf<V>() : pinf<V>();
  for (int q = c + threadIdx.x; q < P; q += RED_NT) {
    val[q] = sent;
    idx[q] = imax_val<I>();
  }
  __syncthreads();
  for (int kk = 2; kk <= P; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += RED_NT) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const bool up = (i & kk) == 0;
          const V vi = val[i], vj = val[ixj];
          const I ii = idx[i], ij = idx[ixj];
          const bool sw = up ? top_before(side, vj, ij, vi, ii) : top_before(side, vi, ii, vj, ij);
          if (sw) {
            val[i] = vj; val[ixj] = vi;
            idx[i] = ij; idx[ixj] = ii;
          }
        }
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) tb.cnt[side] = c < M ? c : M;
  __syncthreads();
}

template <typename V, typename I>
__device__ __forceinline__ V top_threshold(const TopBuf<V, I>& tb, int side, int M) {
  if (tb.cnt[side] >= M) return tb.val[side][M - 1];
  return side == 0 ? -pinf<V>() : pinf<V>();
}

template <typename V, typename I>
__device__ __forceinline__ void top_offer(TopBuf<V, I>& tb, V o, I id, V thr_hi, V thr_lo) {
  if (o >= thr_hi) {
    const int p = atomicAdd(&tb.cnt[0], 1);
    tb.val[0][p] = o;
    tb.idx[0][p] = id;
  }
  if (o <= thr_lo) {
    const int p = atomicAdd(&tb.cnt[1], 1);
    tb.val[1][p] = o;
    tb.idx[1][p] = id;
  }
}

// Write the block's sorted top lists (global ids) to part_top[block][side][M].
template <typename V, typename I>
__device__ void top_write(const TopBuf<V, I>& tb, int M, unsigned long long id_off, TopEnt* dst) {
  for (int side = 0; side < 2; side++) {
    const int c = tb.cnt[side];
    for (int q = threadIdx.x; q < M; q += RED_NT) {
      TopEnt e;
      if (q < c) {
        e.v = (double)tb.val[side][q];
        e.id = (unsigned long long)tb.idx[side][q] + id_off;
      } else {
        e.v = 0.0;
        e.id = ~0ull;
      }
      dst[(size_t)side * M + q] = e;
    }
  }
}

// ---------------------------------------------------------------- shared memory layout
struct SmemLayout {
  size_t binom, R, ls, tv0, tv1, ti0, ti1, total;
};
__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline SmemLayout smem_layout(int N, int k, int ldr, size_t vsz, size_t isz,
                                                  int with_top) {
  SmemLayout L;
  size_t o = 0;
  L.binom = o; o = align16(o + (size_t)(N + 1) * (size_t)(k + 1) * 8);
  L.R = o;     o = align16(o + (size_t)N * (size_t)ldr * vsz);
  L.ls = o;    o = align16(o + (size_t)N * vsz);
  if (with_top) {
    L.tv0 = o; o = align16(o + TOP_CAP * vsz);
    L.tv1 = o; o = align16(o + TOP_CAP * vsz);
    L.ti0 = o; o = align16(o + TOP_CAP * isz);
    L.ti1 = o; o = align16(o + TOP_CAP * isz);
  } else {
    L.tv0 = L.tv1 = L.ti0 = L.ti1 = 0;
  }
  L.total = o;
  return L;
}
__host__ __device__ inline int row_stride(int N) { return N | 1; }

// Load the binomial rows 0..N (columns 0..k), R (FP32 or FP64) and log
// Sigma_ii into shared memory.
template <typename V>
__device__ void load_tables(const NpletArgs& a, unsigned char* smem, const SmemLayout& L,
                            const V* Rg) {
  unsigned long long* sb = reinterpret_cast<unsigned long long*>(smem + L.binom);
  V* sR = reinterpret_cast<V*>(smem + L.R);
  V* sls = reinterpret_cast<V*>(smem + L.ls);
  const int N = a.N, k = a.k, bs = k + 1, ldr = row_stride(N);
  for (int q = threadIdx.x; q < (N + 1) * bs; q += blockDim.x)
    sb[q] = a.binom[(q / bs) * NB + (q % bs)];
  for (int q = threadIdx.x; q < N * N; q += blockDim.x) sR[(q / N) * ldr + (q % N)] = Rg[q];
  for (int q = threadIdx.x; q < N; q += blockDim.x) sls[q] = (V)a.ls[q];
  __syncthreads();
}

// Warp-aggregated append of a global id to an FP64 re-factor list (every
// active lane of the warp appends to the same list).
__device__ __forceinline__ void flag_append_to(unsigned long long* ids, unsigned long long* count,
                                               unsigned long long cap, int* status, bool flag,
                                               unsigned long long id) {
  const unsigned act = __activemask();
  const unsigned fl = __ballot_sync(act, flag);
  if (!fl) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(fl) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(fl));
  if (flag) {
    base = __shfl_sync(fl, base, leader);
    const unsigned long long pos = base + __popc(fl & ((1u << lane) - 1u));
    if (pos < cap) ids[pos] = id;
    else atomicOr(status, ST_FLAG_OVERFLOW);
  }
}
__device__ __forceinline__ void flag_append(const NpletArgs& a, bool flag, unsigned long long id) {
  flag_append_to(a.flag_ids, a.flag_count, a.flag_cap, a.status, flag, id);
}

// Basis store (mode 2): log det R_S, sum_j log p_j and sum_i log Sigma_ii of
// one nplet at out[m * out_n + (gid - out_first)], m = 0, 1, 2, FP32.  A
// flagged nplet (re-factored in FP64 later) stores NaN as its log det.
__device__ __forceinline__ void store_basis(const NpletArgs& a, unsigned long long gid, float lr,
                                            float sp, float lsum, bool flagged) {
  const unsigned long long o = gid - a.out_first;
  float* O = reinterpret_cast<float*>(a.out);
  O[o] = flagged ? __int_as_float(0x7fc00000) : lr;
  O[a.out_n + o] = sp;
  O[2 * a.out_n + o] = lsum;
}

// Per-nplet SoA store (the five measures, or one of them when out_sel > 0).
template <typename V>
__device__ __forceinline__ void store5(const NpletArgs& a, unsigned long long gid, const V (&v)[5]) {
  const unsigned long long o = gid - a.out_first;
  if (a.out_sel > 0) {
    const V x = pick5(v, a.out_sel - 1);
    if (a.out_f64) reinterpret_cast<double*>(a.out)[o] = (double)x;
    else reinterpret_cast<float*>(a.out)[o] = (float)x;
    return;
  }
  if (a.out_f64) {
    double* O = reinterpret_cast<double*>(a.out);
#pragma unroll
    for (int m = 0; m < 5; m++) O[(size_t)m * a.out_n + o] = (double)v[m];
  } else {
    float* O = reinterpret_cast<float*>(a.out);
#pragma unroll
    for (int m = 0; m < 5; m++) O[(size_t)m * a.out_n + o] = (float)v[m];
  }
}

}  // namespace thoi
