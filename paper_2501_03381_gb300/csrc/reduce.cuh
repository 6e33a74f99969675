// Block-level streaming reduction of basis values (shared by the
// single-range and the batched reduction kernels); see reduce.cu.
#pragma once
#include <type_traits>

#include "nplet_common.cuh"

namespace thoi {

constexpr int RB_VEC = 1;                     // 16-byte groups per array per thread per round
constexpr int RB_PER_THREAD = 4 * RB_VEC;     // elements per thread per round
constexpr int RTOP_CAP = 2048;                // candidate buffer per side (>= M + NT * RB)
static_assert(RTOP_CAP >= THOI_MAX_TOP_M + RED_NT * RB_PER_THREAD, "top-M buffer too small");

// Reduction of one range by the calling block (first = the thread's first
// round index, step = rounds advance by this many threads), written to *part
// and part_top[0 .. 2*top_m).  Shared by the single-range kernel (the grid
// strides over one range) and the batched kernel (each block owns tiles).
template <typename V, bool LIST>
__device__ void reduce_core(unsigned long long first, unsigned long long step,
                            const V* __restrict__ blr,
                                                         const V* __restrict__ bsp,
                                                         const V* __restrict__ bls,
                                                         unsigned long long n_dense,
                                                         const unsigned long long* __restrict__ ids,
                                                         const unsigned long long* list_count,
                                                         unsigned long long list_cap,
                                                         unsigned long long id0, Combine cmb,
                                                         int top_m, int nan_is_notpd,
                                                         const float* __restrict__ seed_thr,
                                                         PartRec* __restrict__ part,
                                                         TopEnt* __restrict__ part_top,
                                                         unsigned char* smem, RedScratch& sc,
                                                         int* s_tcnt) {
  using I = typename std::conditional<LIST, unsigned long long, unsigned>::type;
  const bool with_top = top_m > 0;
  TopBuf<V, I> tb;
  tb.val[0] = reinterpret_cast<V*>(smem);
  tb.val[1] = tb.val[0] + RTOP_CAP;
  tb.idx[0] = reinterpret_cast<I*>(tb.val[1] + RTOP_CAP);
  tb.idx[1] = tb.idx[0] + RTOP_CAP;
  tb.cnt = s_tcnt;
  if (threadIdx.x == 0) s_tcnt[0] = s_tcnt[1] = 0;
  __syncthreads();
  V thr_hi = -pinf<V>(), thr_lo = pinf<V>();
  if (seed_thr) {
    thr_hi = (V)seed_thr[0];
    thr_lo = (V)seed_thr[1];
  }
  ThreadRed<V, I> tr;
  tr.init();
  unsigned notpd = 0;
  unsigned long long n = n_dense;
  if (LIST) {
    const unsigned long long c = *list_count;
    n = c < list_cap ? c : list_cap;
  }
  const unsigned long long nq = (n + RB_PER_THREAD - 1) / RB_PER_THREAD;
  const unsigned long long stride = step;
  const unsigned long long rounds = (nq + stride - 1) / stride;
  const int trigger = RTOP_CAP - RED_NT * RB_PER_THREAD;
  const CombineV<V> cmbv(cmb);
  // one round = RB_PER_THREAD elements per thread, loaded as RB_VEC groups of
  // four (all loads of a round are issued together)
  for (unsigned long long rd = 0; rd < rounds; rd++) {
    const unsigned long long q = rd * stride + first;
    if (q < nq) {
      const unsigned long long e0 = q * RB_PER_THREAD;
      V lr[RB_PER_THREAD], sp[RB_PER_THREAD], ls[RB_PER_THREAD];
      unsigned long long pos[RB_PER_THREAD];
#pragma unroll
      for (int t = 0; t < RB_PER_THREAD; t++) pos[t] = e0 + t;
      if (sizeof(V) == 4 && e0 + RB_PER_THREAD <= n) {
#pragma unroll
        for (int g = 0; g < RB_VEC; g++) {
          const float4 fx = reinterpret_cast<const float4*>(blr)[q * RB_VEC + g];
          const float4 fy = reinterpret_cast<const float4*>(bsp)[q * RB_VEC + g];
          const float4 fz = reinterpret_cast<const float4*>(bls)[q * RB_VEC + g];
          lr[4 * g] = fx.x; lr[4 * g + 1] = fx.y; lr[4 * g + 2] = fx.z; lr[4 * g + 3] = fx.w;
          sp[4 * g] = fy.x; sp[4 * g + 1] = fy.y; sp[4 * g + 2] = fy.z; sp[4 * g + 3] = fy.w;
          ls[4 * g] = fz.x; ls[4 * g + 1] = fz.y; ls[4 * g + 2] = fz.z; ls[4 * g + 3] = fz.w;
        }
      } else {
#pragma unroll
        for (int t = 0; t < RB_PER_THREAD; t++) {
          const bool ok = e0 + t < n;
          lr[t] = ok ? blr[e0 + t] : pinf<V>() - pinf<V>();
          sp[t] = ok ? bsp[e0 + t] : (V)0;
          ls[t] = ok ? bls[e0 + t] : (V)0;
        }
      }
#pragma unroll
      for (int t = 0; t < RB_PER_THREAD; t++) {
        if (e0 + t >= n) continue;
        if (is_nan(lr[t])) {
          notpd += nan_is_notpd ? 1u : 0u;
          continue;
        }
        V v[5];
        combine5<V>(lr[t], sp[t], ls[t], cmbv, v);
        if (LIST) {
          const I id = (I)ids[pos[t]];
          tr.add(v, id, lr[t], sp[t], ls[t]);
          if (with_top) top_offer(tb, pick5(v, cmb.top), id, thr_hi, thr_lo);
        } else {
          const I loc = (I)(e0 + t);
          tr.add_mono(v, loc, lr[t], sp[t], ls[t]);
          if (with_top) top_offer(tb, pick5(v, cmb.top), loc, thr_hi, thr_lo);
        }
        if ((t & 3) == 3) tr.flush();
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
      // every thread has read the counts before anyone appends again
      __syncthreads();
    }
  }
  int th = 0, tl = 0;
  const unsigned long long id_off = LIST ? 0ull : id0;
  if (with_top) {
    top_sort_cut(tb, 0, top_m);
    top_sort_cut(tb, 1, top_m);
    th = tb.cnt[0];
    tl = tb.cnt[1];
    top_write(tb, top_m, id_off, part_top);
  }
  block_write_part<V, I>(tr, notpd, id_off, sc, part, th, tl);
}

}  // namespace thoi
