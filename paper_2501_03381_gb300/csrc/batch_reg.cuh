// Batched register-resident FP32 nplet kernel: one persistent launch per
// order k covers the nplets of every dataset of a batch (Methods, "Parallel
// and batched computation of HOI": several datasets evaluated together).
// Block b takes tiles b, b + grid, b + 2 grid, ... of a tile list in which
// every tile is a range of ranks of one (dataset, order) slot; the block
// reloads the dataset's tables (binomial rows, FP32 correlation,
// log-variances) into shared memory when consecutive tiles belong to
// different datasets.  Per nplet the arithmetic is that of the single-
// dataset kernel (nplet_reg_one: LDL^T, unit-lower inverse, inverse
// diagonal); the output is the basis triple of the streaming reduction, and
// flagged nplets are appended to their slot's FP64 re-factor list.
#pragma once
#include "nplet_reg.cuh"

namespace thoi {

__host__ __device__ inline SmemLayout batch_layout(int N, int K) {
  return smem_layout(N, K, row_stride(N), sizeof(float), sizeof(unsigned), 0);
}

template <int K, typename M>
__global__ void __launch_bounds__(RED_NT, RegBlocks<K>::value) k_nplet_reg_batch(const BatchArgs b,
                                                                                const int chunk) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_stop;
  int cur_d = -1, N = 0, ldr = 1;
  float tau_piv = 0.f, tau_tr = 0.f;
  SmemLayout L = batch_layout(1, K);
  for (int t = blockIdx.x; t < b.n_tiles; t += gridDim.x) {
    const BatchTile tile = b.tiles[t];
    const int si = tile.slot;
    const int d = b.slots[si].d;
    const unsigned long long id_base = b.slots[si].id_base;
    const unsigned long long fo = b.slots[si].flag_off, fcap = b.slots[si].flag_cap;
    // every thread is done with the previous tile's tables
    __syncthreads();
    if (threadIdx.x == 0) s_stop = b.cancel ? *(volatile const int*)b.cancel : 0;
    if (d != cur_d) {
      const BatchDataset ds = b.ds[d];
      N = ds.N;
      ldr = row_stride(N);
      tau_piv = ds.tau_piv;
      tau_tr = ds.tau_tr;
      L = batch_layout(N, K);
      unsigned long long* sb = reinterpret_cast<unsigned long long*>(smem + L.binom);
      float* sRw = reinterpret_cast<float*>(smem + L.R);
      float* slw = reinterpret_cast<float*>(smem + L.ls);
      constexpr int bs = K + 1;
      for (int q = threadIdx.x; q < (N + 1) * bs; q += RED_NT)
        sb[q] = b.binom[(q / bs) * NB + (q % bs)];
      for (int q = threadIdx.x; q < N * N; q += RED_NT) sRw[(q / N) * ldr + (q % N)] = ds.R32[q];
      for (int q = threadIdx.x; q < N; q += RED_NT) slw[q] = (float)ds.ls[q];
      cur_d = d;
    }
    __syncthreads();
    if (s_stop) {
      if (threadIdx.x == 0) atomicOr(b.status, ST_CANCELLED);
      break;
    }
    const unsigned long long* sb = reinterpret_cast<const unsigned long long*>(smem + L.binom);
    const float* sR = reinterpret_cast<const float*>(smem + L.R);
    const float* sls = reinterpret_cast<const float*>(smem + L.ls);
    const M full = (N >= (int)(8 * sizeof(M))) ? ~(M)0 : (((M)1 << N) - 1);
    const unsigned n = tile.n;
    const unsigned nch = (n + chunk - 1) / chunk;
    float* B0 = b.basis + tile.boff;
    for (unsigned ch = threadIdx.x; ch < nch; ch += RED_NT) {
      const unsigned e0 = ch * chunk;
      const unsigned long long r0 = tile.r0 + e0;
      const int cnt = n - e0 < (unsigned)chunk ? (int)(n - e0) : chunk;
      M mask = unrank_s<M>(r0, K, N, sb, K + 1);
      for (int j = 0; j < cnt; j++) {
        float lr, sp, lsum, pmin, trace;
        bool bad = false;
        nplet_reg_one<K, M>(mask, N, sR, ldr, sls, lr, sp, lsum, pmin, trace, bad);
        bad |= !(pmin >= tau_piv) | !(trace <= tau_tr);
        const unsigned o = e0 + j;
        B0[o] = bad ? __int_as_float(0x7fc00000) : lr;
        B0[b.bstride + o] = sp;
        B0[2 * b.bstride + o] = lsum;
        flag_append_to(b.flag_ids + fo, b.flag_counts + si, fcap, b.status, bad,
                       id_base + r0 + j);
        if (j + 1 < cnt) mask = lex_succ(mask, full);
      }
    }
  }
}

template <int K, typename M>
static cudaError_t batch_occ_t(int maxN, size_t* smem, int* occ) {
  *smem = batch_layout(maxN, K).total;
  return occupancy_cached((const void*)k_nplet_reg_batch<K, M>, RED_NT, *smem, occ);
}

template <int K>
cudaError_t batch_occ_k(bool wide, int maxN, size_t* smem, int* occ) {
  if (wide) return batch_occ_t<K, unsigned long long>(maxN, smem, occ);
  return batch_occ_t<K, unsigned>(maxN, smem, occ);
}

template <int K>
cudaError_t batch_launch_k(bool wide, const BatchArgs& b, size_t smem, int grid, int chunk,
                           cudaStream_t s) {
  if (wide) k_nplet_reg_batch<K, unsigned long long><<<grid, RED_NT, smem, s>>>(b, chunk);
  else k_nplet_reg_batch<K, unsigned><<<grid, RED_NT, smem, s>>>(b, chunk);
  return cudaGetLastError();
}

#define THOI_BATCH_INSTANCE(KK)                                                              \
  template cudaError_t batch_occ_k<KK>(bool, int, size_t*, int*);                          \
  template cudaError_t batch_launch_k<KK>(bool, const BatchArgs&, size_t, int, int,         \
                                          cudaStream_t);

}  // namespace thoi
