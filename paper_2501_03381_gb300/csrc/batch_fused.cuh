// Persistent batched FP32 nplet kernel with the per-order reduction inside
// (Methods, "Parallel and batched computation of HOI": many datasets
// evaluated together; here of uneven N and T).  One launch covers every
// (dataset, order) slot of a batch whose orders lie in [KLO, KHI]: the
// blocks draw tiles (a range of ranks of one slot) from a device counter, in
// the order of the tile list (largest orders first, so the longest tiles
// start first), and dispatch on the tile's order to a body specialised for
// it.  A block reloads the dataset's tables (binomial rows, FP32
// correlation, log-variances) into shared memory when its next tile belongs
// to another dataset.
//
// Per tile the block evaluates every nplet with the arithmetic of the one-
// thread register kernel (nplet_reg_one: LDL^T, unit-lower inverse, inverse
// diagonal) and reduces in place: each thread keeps min/max with local ids,
// compensated sums and counts, and offers the ranked measure to two top-M
// buffers in shared memory, cut back to M entries between rounds (every
// thread of the block runs the same rounds, so the barriers are uniform).
// The tile's partial record and top lists go to the slot's partial range;
// flagged nplets go to the slot's FP64 re-factor list.  No per-nplet value
// reaches device memory.
#pragma once
#include "nplet_reg.cuh"

namespace thoi {

constexpr int BF_TRIGGER = TOP_CAP - RED_NT * 8;  // cut a top buffer above this count

template <int KHI>
__host__ __device__ inline SmemLayout bfused_layout(int N) {
  return smem_layout(N, KHI, row_stride(N), sizeof(float), sizeof(unsigned), 1);
}

// Reduction of one tile by the whole block.
template <int K, int KHI, typename M>
__device__ __forceinline__ void bfused_tile(const BatchFArgs& b, const BatchFTile& tile,
                                            const BatchSlot& sl, int N, float tau_piv,
                                            float tau_tr, unsigned char* smem,
                                            const SmemLayout& L, RedScratch& sc, int* s_tcnt) {
  constexpr int bs = KHI + 1;
  const unsigned long long* sb = reinterpret_cast<const unsigned long long*>(smem + L.binom);
  const float* sR = reinterpret_cast<const float*>(smem + L.R);
  const float* sls = reinterpret_cast<const float*>(smem + L.ls);
  const int ldr = row_stride(N);
  const int top_m = b.top_m;
  const bool with_top = top_m > 0;
  TopBuf<float, unsigned> tb;
  tb.val[0] = reinterpret_cast<float*>(smem + L.tv0);
  tb.val[1] = reinterpret_cast<float*>(smem + L.tv1);
  tb.idx[0] = reinterpret_cast<unsigned*>(smem + L.ti0);
  tb.idx[1] = reinterpret_cast<unsigned*>(smem + L.ti1);
  tb.cnt = s_tcnt;
  if (threadIdx.x == 0) s_tcnt[0] = s_tcnt[1] = 0;
  __syncthreads();
  // start from the tightest bounds the slot's finished tiles have published
  // (the M-th best of any subset bounds the M-th best of the slot)
  float thr_hi = -pinf<float>(), thr_lo = pinf<float>();
  if (with_top && b.slot_thr) {
    const unsigned khi = b.slot_thr[2 * tile.slot], klo = b.slot_thr[2 * tile.slot + 1];
    if (khi) thr_hi = fkey32_value(khi);
    if (klo) thr_lo = fkey32_value(~klo);
  }
  // a cut keeps the tighter of the tile's own M-th best and the slot's bound,
  // and publishes it for the slot's other tiles
  auto publish = [&]() {
    if (threadIdx.x == 0 && b.slot_thr) {
      if (thr_hi > -pinf<float>()) atomicMax(&b.slot_thr[2 * tile.slot], fkey32(thr_hi));
      if (thr_lo < pinf<float>()) atomicMax(&b.slot_thr[2 * tile.slot + 1], ~fkey32(thr_lo));
    }
  };
  ThreadRed<float, unsigned> tr;
  tr.init();
  const CombineV<float> cmbv(sl.cmb);
  const int rank_m = sl.cmb.top;
  const M full = (N >= (int)(8 * sizeof(M))) ? ~(M)0 : (((M)1 << N) - 1);
  const int chunk = b.chunk_k[K];
  const unsigned nch = (tile.n + chunk - 1) / chunk;
  const unsigned rounds = (nch + RED_NT - 1) / RED_NT;
  const unsigned long long id_off = sl.id_base + tile.r0;
  unsigned long long* fids = b.flag_ids + sl.flag_off;
  unsigned long long* fcnt = b.flag_counts + tile.slot;
  for (unsigned rd = 0; rd < rounds; rd++) {
    const unsigned ch = rd * RED_NT + threadIdx.x;
    if (ch < nch) {
      const unsigned e0 = ch * chunk;
      const int cnt = tile.n - e0 < (unsigned)chunk ? (int)(tile.n - e0) : chunk;
      M mask = unrank_s<M>(tile.r0 + e0, K, N, sb, bs);
      for (int j = 0; j < cnt; j++) {
        float lr, sp, lsum, pmin, trace;
        bool bad = false;
        nplet_reg_one<K, M>(mask, N, sR, ldr, sls, lr, sp, lsum, pmin, trace, bad);
        bad |= !(pmin >= tau_piv) | !(trace <= tau_tr);
        const unsigned loc = e0 + j;
        if (!bad) {
          float v[5];
          combine5<float>(lr, sp, lsum, cmbv, v);
          tr.add_mono(v, loc, lr, sp, lsum);
          if (with_top) top_offer(tb, pick5(v, rank_m), loc, thr_hi, thr_lo);
        }
        flag_append_to(fids, fcnt, sl.flag_cap, b.status, bad, id_off + loc);
        if (j + 1 < cnt) mask = lex_succ(mask, full);
      }
    }
    if (with_top) {
      __syncthreads();
      const bool c0 = tb.cnt[0] > BF_TRIGGER, c1 = tb.cnt[1] > BF_TRIGGER;
      if (c0) {
        top_sort_cut(tb, 0, top_m);
        thr_hi = fmaxf(thr_hi, top_threshold(tb, 0, top_m));
      }
      if (c1) {
        top_sort_cut(tb, 1, top_m);
        thr_lo = fminf(thr_lo, top_threshold(tb, 1, top_m));
      }
      if (c0 | c1) publish();
      __syncthreads();
    }
  }
  int th = 0, tl = 0;
  if (with_top) {
    top_sort_cut(tb, 0, top_m);
    top_sort_cut(tb, 1, top_m);
    th = tb.cnt[0];
    tl = tb.cnt[1];
    thr_hi = fmaxf(thr_hi, top_threshold(tb, 0, top_m));
    thr_lo = fminf(thr_lo, top_threshold(tb, 1, top_m));
    publish();
    top_write(tb, top_m, id_off, b.part_top + (size_t)tile.pidx * 2 * top_m);
  }
  block_write_part<float, unsigned>(tr, 0u, id_off, sc, b.part + tile.pidx, th, tl);
}

template <int K, int KHI, typename M>
struct BfDispatch {
  __device__ __forceinline__ static void run(int k, const BatchFArgs& b, const BatchFTile& tile,
                                             const BatchSlot& sl, int N, float tp, float tt,
                                             unsigned char* smem, const SmemLayout& L,
                                             RedScratch& sc, int* s_tcnt) {
    if (k == K) bfused_tile<K, KHI, M>(b, tile, sl, N, tp, tt, smem, L, sc, s_tcnt);
    else BfDispatch<K + 1, KHI, M>::run(k, b, tile, sl, N, tp, tt, smem, L, sc, s_tcnt);
  }
};
template <int KHI, typename M>
struct BfDispatch<KHI + 1, KHI, M> {
  __device__ __forceinline__ static void run(int, const BatchFArgs&, const BatchFTile&,
                                             const BatchSlot&, int, float, float, unsigned char*,
                                             const SmemLayout&, RedScratch&, int*) {}
};

// Minimum resident blocks per SM: the bodies of the band's largest order
// bound the registers.
template <int KHI>
struct BfBlocks {
  static constexpr int value = KHI <= 8 ? 4 : (KHI <= 14 ? 3 : 2);
};

template <int KLO, int KHI, typename M>
__global__ void __launch_bounds__(RED_NT, BfBlocks<KHI>::value) k_batch_fused(const BatchFArgs b) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ RedScratch sc;
  __shared__ int s_tcnt[2];
  __shared__ int s_tile, s_stop;
  int cur_d = -1, N = 1;
  float tau_piv = 0.f, tau_tr = 0.f;
  SmemLayout L = bfused_layout<KHI>(1);
  for (;;) {
    // every thread is done with the previous tile's tables and buffers
    __syncthreads();
    if (threadIdx.x == 0) {
      s_tile = (int)atomicAdd(b.tile_counter, 1u);
      s_stop = b.cancel ? *(volatile const int*)b.cancel : 0;
    }
    __syncthreads();
    const int t = s_tile;
    if (t >= b.n_tiles) break;
    if (s_stop) {
      if (threadIdx.x == 0) atomicOr(b.status, ST_CANCELLED);
      break;
    }
    const BatchFTile tile = b.tiles[t];
    const BatchSlot sl = b.slots[tile.slot];
    if (sl.d != cur_d) {
      const BatchDataset ds = b.ds[sl.d];
      N = ds.N;
      tau_piv = ds.tau_piv;
      tau_tr = ds.tau_tr;
      L = bfused_layout<KHI>(N);
      const int ldr = row_stride(N);
      constexpr int bs = KHI + 1;
      unsigned long long* sbw = reinterpret_cast<unsigned long long*>(smem + L.binom);
      float* sRw = reinterpret_cast<float*>(smem + L.R);
      float* slw = reinterpret_cast<float*>(smem + L.ls);
      for (int q = threadIdx.x; q < (N + 1) * bs; q += RED_NT)
        sbw[q] = b.binom[(q / bs) * NB + (q % bs)];
      for (int q = threadIdx.x; q < N * N; q += RED_NT) sRw[(q / N) * ldr + (q % N)] = ds.R32[q];
      for (int q = threadIdx.x; q < N; q += RED_NT) slw[q] = (float)ds.ls[q];
      cur_d = sl.d;
      // the tile body's first barrier orders these stores before any read
    }
    BfDispatch<KLO, KHI, M>::run(tile.k, b, tile, sl, N, tau_piv, tau_tr, smem, L, sc, s_tcnt);
  }
}

template <int KLO, int KHI>
cudaError_t bfused_launch(bool wide, const BatchFArgs& b, int maxN, int blocks_per_sm,
                          int num_sms, cudaStream_t s, int* grid_out) {
  const size_t sm = bfused_layout<KHI>(maxN).total;
  const void* fn = wide ? (const void*)k_batch_fused<KLO, KHI, unsigned long long>
                        : (const void*)k_batch_fused<KLO, KHI, unsigned>;
  int occ = 0;
  cudaError_t e = occupancy_cached(fn, RED_NT, sm, &occ);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  if (blocks_per_sm > 0 && blocks_per_sm < occ) occ = blocks_per_sm;
  long long grid = (long long)num_sms * occ;
  if (grid > b.n_tiles) grid = b.n_tiles;
  if (grid < 1) grid = 1;
  if (wide) k_batch_fused<KLO, KHI, unsigned long long><<<(unsigned)grid, RED_NT, sm, s>>>(b);
  else k_batch_fused<KLO, KHI, unsigned><<<(unsigned)grid, RED_NT, sm, s>>>(b);
  if (grid_out) *grid_out = (int)grid;
  return cudaGetLastError();
}

}  // namespace thoi
