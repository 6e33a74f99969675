// Register-resident FP32 nplet kernel for orders too large for one thread's
// registers: a group of G consecutive lanes shares one nplet.  Row i of the
// k x k correlation submatrix (lower triangle) lives in the registers of lane
// i mod G, so each lane holds about k^2 / (2G) entries.
//
// Per nplet (same quantities as the one-thread kernel):
//   Cholesky, right-looking: step p broadcasts the pivot and the scaled
//     column p inside the group (shuffles); each lane updates its own rows.
//   Triangular inverse W = L^-1, right-looking by rows: row m of W is
//     finished by its owner, broadcast, and subtracted (times L_im) from the
//     lanes' rows i > m; rows are stored in place of L.
//   (R_S^-1)_jj = sum_i W_ij^2: per-lane partial column sums, then a
//     butterfly over the group.
// Every lane of a group computes the pivots and the column norms, so the
// products, the smallest pivot and the trace are identical in all of them;
// lane 0 of the group does the reduction, output and flagging.
#pragma once
#include "nplet_common.cuh"

namespace thoi {

template <int K, int G>
__device__ __forceinline__ void chol_loo_grp(float (&A)[(K + G - 1) / G][K], int g, int gbase,
                                             unsigned gmask, float& lr, float& sp, float& pmin,
                                             float& trace, bool& bad) {
  constexpr int R = (K + G - 1) / G;
  float P1 = 1.f, P2 = 1.f;
  int E1 = 0, E2 = 0;
  pmin = pinf<float>();
  // ---------------- Cholesky
#pragma unroll
  for (int p = 0; p < K; p++) {
    const float d = __shfl_sync(gmask, A[p / G][p], gbase + p % G);
    pmin = fminf(pmin, d);
    P1 *= d;
    if ((p & 3) == 3 || p == K - 1) renorm(P1, E1, bad);
    const float inv = rsqrtf(d);
    if (g == p % G) A[p / G][p] = inv;
    // scale the lane's own entries of column p below the diagonal
#pragma unroll
    for (int r = 0; r < R; r++) {
      if (r * G + G - 1 <= p) continue;  // no row of this block lies below p
      const int i = r * G + g;
      if (i > p && i < K) A[r][p] *= inv;
    }
    // broadcast the scaled column p
    float col[K];
#pragma unroll
    for (int j = p + 1; j < K; j++) col[j] = __shfl_sync(gmask, A[j / G][p], gbase + j % G);
    // trailing update of the lane's rows
#pragma unroll
    for (int r = 0; r < R; r++) {
      if (r * G + G - 1 <= p) continue;
      const int i = r * G + g;
      const bool row_ok = i > p && i < K;
#pragma unroll
      for (int j = p + 1; j < K && j <= r * G + G - 1; j++) {
        if (row_ok && j <= i) A[r][j] = fmaf(-A[r][p], col[j], A[r][j]);
      }
    }
  }
  // ---------------- W = L^-1 by rows, in place
#pragma unroll
  for (int m = 0; m < K; m++) {
    const int om = m % G, mr = m / G;
    // the owner finishes row m: W_mc = T_mc / L_mm (W_mm = 1/L_mm is stored)
    if (g == om) {
#pragma unroll
      for (int c = 0; c < m; c++) A[mr][c] *= A[mr][m];
    }
    float w[K];
#pragma unroll
    for (int c = 0; c <= m; c++) w[c] = __shfl_sync(gmask, A[mr][c], gbase + om);
#pragma unroll
    for (int r = 0; r < R; r++) {
      if (r * G + G - 1 <= m) continue;
      const int i = r * G + g;
      if (i > m && i < K) {
        const float lim = A[r][m];
        A[r][m] = -lim * w[m];
#pragma unroll
        for (int c = 0; c < m; c++) A[r][c] = fmaf(-lim, w[c], A[r][c]);
      }
    }
  }
  // ---------------- p_j = sum_i W_ij^2
  float ps[K];
#pragma unroll
  for (int c = 0; c < K; c++) ps[c] = 0.f;
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int i = r * G + g;
#pragma unroll
    for (int c = 0; c < K && c <= r * G + G - 1; c++)
      if (c <= i && i < K) ps[c] = fmaf(A[r][c], A[r][c], ps[c]);
  }
  trace = 0.f;
#pragma unroll
  for (int c = 0; c < K; c++) {
#pragma unroll
    for (int o = 1; o < G; o <<= 1) ps[c] += __shfl_xor_sync(gmask, ps[c], o);
    trace += ps[c];
    P2 *= ps[c];
    if ((c & 3) == 3 || c == K - 1) renorm(P2, E2, bad);
  }
  lr = log_of(P1, E1);
  sp = log_of(P2, E2);
}

template <int K, int G, typename M>
__global__ void __launch_bounds__(RED_NT) k_nplet_grp(const NpletArgs a, const int chunk) {
  constexpr int R = (K + G - 1) / G;
  constexpr int GPB = RED_NT / G;  // groups per block
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = a.N, ldr = row_stride(N);
  const SmemLayout L = smem_layout(N, K, ldr, sizeof(float), sizeof(unsigned), 0);
  load_tables<float>(a, smem, L, a.R32);
  const unsigned long long* sb = reinterpret_cast<const unsigned long long*>(smem + L.binom);
  const float* sR = reinterpret_cast<const float*>(smem + L.R);
  const float* sls = reinterpret_cast<const float*>(smem + L.ls);
  const bool basis = a.mode == 2;
  const bool fused = a.mode == 3;
  const float* sthr = reinterpret_cast<const float*>(smem + L.thr);
  FusedAcc acc;
  acc.init();
  const int lane = threadIdx.x & 31;
  const int g = lane % G;
  const int gbase = lane - g;
  const unsigned gmask = ((1u << G) - 1u) << gbase;
  const bool leader = g == 0;
  const M full = (N >= (int)(8 * sizeof(M))) ? ~(M)0 : (((M)1 << N) - 1);
  const unsigned long long n = a.rank_end - a.rank_begin;
  const unsigned long long nch = (n + chunk - 1) / chunk;
  const unsigned long long stride = (unsigned long long)gridDim.x * GPB;
  const float tau_piv = a.tau_piv, tau_tr = a.tau_tr;
  const CombineV<float> cmbv(a.cmb);

  for (unsigned long long ch = (unsigned long long)blockIdx.x * GPB + threadIdx.x / G; ch < nch;
       ch += stride) {
    // the cancel flag lives in host memory: the leader reads it once every
    // 64 rounds and the whole group follows its answer
    if (((ch / stride) & 63) == 0 && a.cancel) {
      int stop = leader ? *(volatile const int*)a.cancel : 0;
      stop = __shfl_sync(gmask, stop, gbase);
      if (stop) {
        if (leader) atomicOr(a.status, ST_CANCELLED);
        break;
      }
    }
    const unsigned long long r0 = a.rank_begin + ch * chunk;
    const unsigned long long left = a.rank_end - r0;
    const int cnt = left < (unsigned long long)chunk ? (int)left : chunk;
    M mask = unrank_s<M>(r0, K, N, sb, K + 1);
    for (int jn = 0; jn < cnt; jn++) {
      // indices of the nplet; row offsets of the lane's own rows
      int c[K];
      int ro[R];
      {
        M m = mask;
#pragma unroll
        for (int q = 0; q < K; q++) {
          const int hb = hibit(m);
          m ^= (M)1 << hb;
          c[q] = N - 1 - hb;
        }
#pragma unroll
        for (int r = 0; r < R; r++) ro[r] = 0;
#pragma unroll
        for (int q = 0; q < K; q++)
          if (q % G == g) ro[q / G] = c[q] * ldr;
      }
      float A[R][K];
      float lsum = 0.f;
#pragma unroll
      for (int q = 0; q < K; q++) lsum += sls[c[q]];
#pragma unroll
      for (int r = 0; r < R; r++) {
        const int i = r * G + g;
#pragma unroll
        for (int j = 0; j < K && j <= r * G + G - 1; j++)
          A[r][j] = (j <= i && i < K) ? sR[ro[r] + c[j]] : 0.f;
      }
      float lr, sp, pmin, trace;
      bool bad = false;
      chol_loo_grp<K, G>(A, g, gbase, gmask, lr, sp, pmin, trace, bad);
      bad |= !(pmin >= tau_piv) | !(trace <= tau_tr);
      if (leader) {
        const unsigned long long gid = a.id_base + r0 + jn;
        if (fused) {
          fused_emit(a, acc, sthr, cmbv, gid, lr, sp, lsum, bad);
        } else {
          if (basis) {
            store_basis(a, gid, lr, sp, lsum, bad);
          } else {
            float v[5];
            combine5<float>(lr, sp, lsum, cmbv, v);
            store5<float>(a, gid, v);
          }
          flag_append(a, bad, gid);
        }
      }
      if (jn + 1 < cnt) mask = lex_succ(mask, full);
    }
  }
  if (fused) fused_block_end(a, acc);
}

template <int K, int G, typename M>
static cudaError_t launch_grp_t(const NpletArgs& a, const Shape& sh, int num_sms, cudaStream_t s,
                                int* grid_out, int max_blocks) {
  constexpr int GPB = RED_NT / G;
  const SmemLayout L = smem_layout(a.N, K, row_stride(a.N), sizeof(float), sizeof(unsigned), 0);
  void (*fn)(const NpletArgs, const int) = k_nplet_grp<K, G, M>;
  int occ = 0;
  cudaError_t e = occupancy_cached((const void*)fn, RED_NT, L.total, &occ);
  if (e != cudaSuccess) return e;
  if (sh.blocks_per_sm > 0 && sh.blocks_per_sm < occ) occ = sh.blocks_per_sm;
  int chunk = sh.chunk > 0 ? sh.chunk : 4;
  if (chunk > 8) chunk = 8;
  long long grid = (long long)num_sms * occ;
  const unsigned long long n = a.rank_end - a.rank_begin;
  const long long need = (long long)((n + (unsigned long long)GPB * chunk - 1) /
                                     ((unsigned long long)GPB * chunk));
  if (need < grid) grid = need > 0 ? need : 1;
  if (grid > max_blocks) grid = max_blocks;
  fn<<<(unsigned)grid, RED_NT, L.total, s>>>(a, chunk);
  if (grid_out) *grid_out = (int)grid;
  return cudaGetLastError();
}

template <int K, int G>
cudaError_t launch_grp_k(const NpletArgs& a, const Shape& sh, int num_sms, cudaStream_t s,
                         int* grid_out, int max_blocks) {
  if (a.N <= 32) return launch_grp_t<K, G, unsigned>(a, sh, num_sms, s, grid_out, max_blocks);
  return launch_grp_t<K, G, unsigned long long>(a, sh, num_sms, s, grid_out, max_blocks);
}

}  // namespace thoi
