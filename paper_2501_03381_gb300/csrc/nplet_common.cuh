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

// Positive-definiteness of a pivot of the unit-diagonal correlation
// submatrix.  In FP64 a pivot at or below 2^-45 is within the rounding of
// the zero pivot of an exactly singular submatrix (two equal variables, say),
// so it counts as not positive definite whatever its sign; every FP64 kernel
// decides the same way.  FP32 pivots only need to be positive here: small
// ones are flagged for the FP64 re-factor by the pivot threshold.
constexpr double PD_FLOOR64 = 2.8421709430404007e-14;  // 2^-45
constexpr double PD_RCP_CEIL64 = 35184372088832.0;     // 2^45 (bound on 1/D)
__device__ __forceinline__ bool pivot_ok(double d) { return d > PD_FLOOR64; }
__device__ __forceinline__ bool pivot_ok(float d) { return d > 0.f; }
// the same test on a reciprocal pivot 1/D (also rejects 1/0 and NaN)
__device__ __forceinline__ bool rcp_pivot_ok(double rd) {
  return (rd > 0.0) & (rd < PD_RCP_CEIL64);
}

// Reciprocal by the hardware approximation (about 1 ulp), one instruction.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// The final product is rounded on its own (__fmul_rn): left to the compiler,
// a consumer's addition could fuse with it in one kernel and not in another,
// and the records of every path must agree bit for bit.
__device__ __forceinline__ float log_of(float P, int E) {
  return __fmul_rn(__log2f(P) + (float)E, (float)LN2);
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

// Explicit multiply-adds, so that every kernel forms the five values with
// the same roundings (left to the compiler, contraction may differ between
// call sites, and the batched and single-dataset records must agree bit for
// bit).
__device__ __forceinline__ float fma_v(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_v(double a, double b, double c) { return fma(a, b, c); }
template <typename V>
__device__ __forceinline__ void combine5(V lr, V sp, V lsum, const CombineV<V>& c, V (&v)[5]) {
  const V tc = fma_v((V)(-0.5), lr, c.tc_c);
  const V dtc = fma_v((V)0.5, lr + sp, c.dtc_c);
  v[0] = fma_v((V)0.5, lr + lsum, c.h_c);
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

// ---------------------------------------------------------------- fused records (mode 3)
// The per-order reduction done inside the nplet kernels.  Before the order's
// nplet launch a sample kernel bounds every extreme from a sample of the
// order's nplets (the sample's minimum and maximum of each measure, and for
// the ranked measure the smallest block maximum and the largest block
// minimum, so that at least one sampled nplet per sample block lies beyond
// each top-list bound).  The nplet kernel then keeps per thread only the
// compensated sums and the count of O < 0, and appends to a candidate list
// the nplets that lie beyond a bound; the list is reduced like a re-factor
// list.  Every bound is widened by a margin above the FP32 error of a nplet,
// and the merge certifies the final record against the bounds (an extreme
// inside a bound, or a full top list ending beyond it, shows that no nplet
// left off the list could change the record); a record that cannot be
// certified makes the host repeat the order with stored basis values.
__device__ __forceinline__ unsigned fkey32(float v) {
  unsigned u = __float_as_uint(v);
  if ((u << 1) == 0) u = 0;
  return (u >> 31) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey32_value(unsigned k) {
  return __uint_as_float((k >> 31) ? (k & 0x7fffffffu) : ~k);
}
// Whether threshold slot j stores the complement of its key (so that every
// slot is aggregated with atomicMax): the minima of the measures and the
// largest-side top bound (a minimum over sample blocks).
__host__ __device__ __forceinline__ bool fused_slot_negated(int j, int top) {
  return j < 5 ? (j != top) : (j - 5 == top);
}
// Margin added to a bound: a sampled nplet evaluated by another FP32 kernel
// than the one that evaluates it in the order's pass may differ by twice the
// FP32 error of a nplet (at most 1e-4 nats each for the nplets the FP32 path
// keeps), so 5e-4 plus a relative 4e-6 keeps the sampled witnesses beyond
// the bound.
__host__ __device__ __forceinline__ float fused_margin(float t) {
  return 5e-4f + 4e-6f * fabsf(t);
}
// Slot j's bound as a float, widened; a missing bound admits everything.
__device__ __forceinline__ float fused_threshold(unsigned key, int j, int top) {
  const bool le = j < 5;
  if (key == 0u) return le ? pinf<float>() : -pinf<float>();
  const float t = fkey32_value(fused_slot_negated(j, top) ? ~key : key);
  return le ? t + fused_margin(t) : t - fused_margin(t);
}

// ---------------------------------------------------------------- shared memory layout
struct SmemLayout {
  size_t binom, R, ls, thr, tv0, tv1, ti0, ti1, total;
};
__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline SmemLayout smem_layout(int N, int k, int ldr, size_t vsz, size_t isz,
                                                  int with_top) {
  SmemLayout L;
  size_t o = 0;
  L.binom = o; o = align16(o + (size_t)(N + 1) * (size_t)(k + 1) * 8);
  L.R = o;     o = align16(o + (size_t)N * (size_t)ldr * vsz);
  L.ls = o;    o = align16(o + (size_t)N * vsz);
  L.thr = o;   o = align16(o + (size_t)FUSE_NTHR * sizeof(float));
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
  if (a.mode == 3 && threadIdx.x < FUSE_NTHR)
    reinterpret_cast<float*>(smem + L.thr)[threadIdx.x] =
        fused_threshold(a.thr_keys[threadIdx.x], threadIdx.x, a.cmb.top);
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

// ---------------------------------------------------------------- fused records: per nplet
// Per-thread state of the fused records: compensated FP32 sums of the three
// basis values and the count of O < 0 over the nplets the FP32 path keeps.
struct FusedAcc {
  float slr, ssp, sls, clr, csp, cls;
  unsigned neg;
  __device__ __forceinline__ void init() {
    slr = ssp = sls = clr = csp = cls = 0.f;
    neg = 0;
  }
  __device__ __forceinline__ static void kahan(float& s, float& c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

// Warp-aggregated append of one nplet (id and basis values) to the
// candidate list, starting at the block's segment. Entries that do not fit
// go on to the next segment: a kernel that takes its work dynamically may
// leave most candidates to a few blocks. Only a full list raises
// ST_CAND_OVERFLOW (the order is then redone with stored basis values).
__device__ __forceinline__ void cand_append(const NpletArgs& a, bool cand, unsigned long long gid,
                                            float lr, float sp, float lsum) {
  const unsigned act = __activemask();
  unsigned fl = __ballot_sync(act, cand);
  if (!fl) return;
  const int lane = threadIdx.x & 31;
  int seg = (int)(blockIdx.x % (unsigned)a.cand_nseg);
  // fl, t and seg are the same in every lane of act: the loop is warp-uniform
  for (int t = 0; t < a.cand_nseg && fl; t++) {
    const int leader = __ffs(fl) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(a.cand_count + seg, (unsigned long long)__popc(fl));
    base = __shfl_sync(act, base, leader);
    bool left = false;
    if ((fl >> lane) & 1u) {
      const unsigned long long pos = base + __popc(fl & ((1u << lane) - 1u));
      if (pos < a.cand_seg) {
        const unsigned long long e = (unsigned long long)seg * a.cand_seg + pos;
        a.cand_ids[e] = gid;
        a.cand_b[e] = lr;
        a.cand_b[a.cand_cap + e] = sp;
        a.cand_b[2 * a.cand_cap + e] = lsum;
      } else {
        left = true;
      }
    }
    fl = __ballot_sync(act, left);
    seg = seg + 1 == a.cand_nseg ? 0 : seg + 1;
  }
  if ((fl >> lane) & 1u) atomicOr(a.status, ST_CAND_OVERFLOW);
}

// Mode 4: a block's extremes of sampled nplets into the slot's bound keys
// (every thread passes its own minima and maxima; see launch_fused_sample).
__device__ inline void sample_block_keys(const NpletArgs& a, float (&mn)[5], float (&mx)[5],
                                         unsigned valid) {
  __shared__ float s_mn[RED_NT / 32][5], s_mx[RED_NT / 32][5];
  __shared__ unsigned s_valid[RED_NT / 32];
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
    for (int q = 0; q < RED_NT / 32; q++) {
      nv += s_valid[q];
      for (int m = 0; m < 5; m++) {
        mn[m] = fminf(mn[m], s_mn[q][m]);
        mx[m] = fmaxf(mx[m], s_mx[q][m]);
      }
    }
    if (nv > 0) {
      unsigned* keys = const_cast<unsigned*>(a.thr_keys);
      const int top = a.cmb.top;
      for (int m = 0; m < 5; m++) {
        const unsigned klo = fkey32(mn[m]), khi = fkey32(mx[m]);
        atomicMax(&keys[m], fused_slot_negated(m, top) ? ~klo : klo);
        atomicMax(&keys[5 + m], fused_slot_negated(5 + m, top) ? ~khi : khi);
      }
    }
  }
}

// Rank of sample i of S spread evenly over the range (n = q S + rem).
__device__ __forceinline__ unsigned long long sample_rank(const NpletArgs& a, unsigned long long i,
                                                          unsigned long long S) {
  const unsigned long long n = a.rank_end - a.rank_begin;
  const unsigned long long q = n / S, rem = n % S;
  return a.rank_begin + i * q + (i * rem) / S;
}

// One nplet in mode 3: sums and count of O < 0 when the FP32 value is kept,
// candidate test against the block's bounds (sthr, shared memory), and the
// FP64 re-factor list for a flagged nplet.
__device__ __forceinline__ void fused_emit(const NpletArgs& a, FusedAcc& acc, const float* sthr,
                                           const CombineV<float>& cv, unsigned long long gid,
                                           float lr, float sp, float lsum, bool bad) {
  bool cand = false;
  if (!bad) {
    float v[5];
    combine5<float>(lr, sp, lsum, cv, v);
    FusedAcc::kahan(acc.slr, acc.clr, lr);
    FusedAcc::kahan(acc.ssp, acc.csp, sp);
    FusedAcc::kahan(acc.sls, acc.cls, lsum);
    acc.neg += v[3] < 0.f ? 1u : 0u;
#pragma unroll
    for (int m = 0; m < 5; m++) cand |= (v[m] <= sthr[m]) | (v[m] >= sthr[5 + m]);
  }
  cand_append(a, cand, gid, lr, sp, lsum);
  flag_append(a, bad, gid);
}

// End of a mode-3 kernel (every thread of the block): the block's sums and
// count of O < 0 into its partial record; extremes and top lists stay empty
// (they come from the candidate list) and the count is carried by the
// candidate reduction.
__device__ inline void fused_block_end(const NpletArgs& a, const FusedAcc& acc) {
  __shared__ double s_sum[RED_NT / 32][3];
  __shared__ unsigned s_neg[RED_NT / 32];
  double x0 = (double)acc.slr - (double)acc.clr, x1 = (double)acc.ssp - (double)acc.csp,
         x2 = (double)acc.sls - (double)acc.cls;
  unsigned ng = acc.neg;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    x0 += __shfl_xor_sync(0xffffffffu, x0, o);
    x1 += __shfl_xor_sync(0xffffffffu, x1, o);
    x2 += __shfl_xor_sync(0xffffffffu, x2, o);
    ng += __shfl_xor_sync(0xffffffffu, ng, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_sum[w][0] = x0;
    s_sum[w][1] = x1;
    s_sum[w][2] = x2;
    s_neg[w] = ng;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    PartRec r;
    for (int m = 0; m < 5; m++) {
      r.vmin[m] = pinf<double>();
      r.vmax[m] = -pinf<double>();
      r.imin[m] = r.imax[m] = ~0ull;
    }
    r.s_lr = r.s_sp = r.s_ls = 0.0;
    unsigned long long neg = 0;
    for (int q = 0; q < RED_NT / 32; q++) {
      r.s_lr += s_sum[q][0];
      r.s_sp += s_sum[q][1];
      r.s_ls += s_sum[q][2];
      neg += s_neg[q];
    }
    r.count = 0;
    r.neg = neg;
    r.notpd = 0;
    r.top_hi = r.top_lo = 0;
    a.part[blockIdx.x] = r;
  }
}

}  // namespace thoi
