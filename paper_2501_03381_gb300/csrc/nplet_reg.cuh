// Register-resident FP32 nplet kernel (templates), one template instance per order
// k <= 20: each thread owns one nplet at a time, its k x k correlation
// submatrix lives in registers (packed lower triangle), and the Cholesky
// factor, the triangular inverse and the leave-one-out diagonal are computed
// in place with fully unrolled loops (Methods, "Parallel and batched
// computation of HOI": determinants of every submatrix and of every
// leave-one-out submatrix; here logdet R_S + log (R_S^-1)_jj gives the latter).
#pragma once
#include "nplet_common.cuh"

namespace thoi {


// R_S = Lh D Lh^T (Lh unit lower, D the Cholesky pivots), in place: the
// strictly lower part of A becomes Lh, the diagonal 1/D.  Then
// V = -(Lh^-1 - I) column by column (unit lower inverse, FMAs only), and
// p_j = (R_S^-1)_jj = sum_i (Lh^-1)_ij^2 / D_i = 1/D_j + sum_{i>j} V_ij^2 / D_i.
// log det R_S = sum_p log D_p.
template <int K>
__device__ __forceinline__ void chol_loo_reg(float (&A)[K][K], float& lr, float& sp,
                                             float& pmin, float& trace, bool& bad) {
  float P1 = 1.f, P2 = 1.f;
  int E1 = 0, E2 = 0;
  pmin = pinf<float>();
#pragma unroll
  for (int p = 0; p < K; p++) {
    const float d = A[p][p];
    pmin = fminf(pmin, d);
    P1 *= d;
    if ((p & 3) == 3 || p == K - 1) renorm(P1, E1, bad);
    const float rd = rcp_approx(d);
    A[p][p] = rd;
    float u[K];
#pragma unroll
    for (int i = p + 1; i < K; i++) u[i] = A[i][p] * rd;
#pragma unroll
    for (int i = p + 1; i < K; i++)
#pragma unroll
      for (int j = p + 1; j <= i; j++) A[i][j] = fmaf(-u[i], A[j][p], A[i][j]);
#pragma unroll
    for (int i = p + 1; i < K; i++) A[i][p] = u[i];
  }
  trace = 0.f;
#pragma unroll
  for (int j = 0; j < K; j++) {
    float pj = A[j][j];
#pragma unroll
    for (int i = j + 1; i < K; i++) {
      float s = A[i][j];
#pragma unroll
      for (int m = j + 1; m < i; m++) s = fmaf(-A[i][m], A[m][j], s);
      A[i][j] = s;
      pj = fmaf(s * A[i][i], s, pj);
    }
    trace += pj;
    P2 *= pj;
    if ((j & 3) == 3 || j == K - 1) renorm(P2, E2, bad);
  }
  lr = log_of(P1, E1);
  sp = log_of(P2, E2);
}

template <int K, typename M>
__device__ __forceinline__ void nplet_reg_one(M mask, int N, const float* sR, int ldr,
                                              const float* sls, float& lr, float& sp, float& lsum,
                                              float& pmin, float& trace, bool& bad) {
  int c[K];
  M m = mask;
#pragma unroll
  for (int i = 0; i < K; i++) {
    const int hb = hibit(m);
    m ^= (M)1 << hb;
    c[i] = N - 1 - hb;
  }
  // K x K array (only the lower triangle is used): the compiler keeps a
  // two-dimensional array in registers where a packed one of the same
  // size is demoted to local memory.
  float A[K][K];
  lsum = 0.f;
#pragma unroll
  for (int i = 0; i < K; i++) {
    const float* row = sR + c[i] * ldr;
    lsum += sls[c[i]];
#pragma unroll
    for (int j = 0; j <= i; j++) A[i][j] = row[c[j]];
  }
  chol_loo_reg<K>(A, lr, sp, pmin, trace, bad);
}

// Thread t of block b handles, in round r, the chunk of `chunk` consecutive
// lexicographic ranks starting at rank_begin + ((r*G + b)*NT + t)*chunk:
// neighbouring threads hold neighbouring nplets, which share most indices,
// so their shared-memory gathers mostly hit the same words.
template <int K, typename M>
__global__ void __launch_bounds__(RED_NT) k_nplet_reg(const NpletArgs a, const int chunk) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ RedScratch sc;
  __shared__ int s_tcnt[2];
  __shared__ int s_stop;
  const int N = a.N, ldr = row_stride(N);
  const bool red = a.mode == 1;
  const bool with_top = red && a.top_m > 0;
  const SmemLayout L = smem_layout(N, K, ldr, sizeof(float), sizeof(unsigned), with_top);
  if (threadIdx.x == 0) { s_tcnt[0] = s_tcnt[1] = 0; s_stop = 0; }
  load_tables<float>(a, smem, L, a.R32);
  const unsigned long long* sb = reinterpret_cast<const unsigned long long*>(smem + L.binom);
  const float* sR = reinterpret_cast<const float*>(smem + L.R);
  const float* sls = reinterpret_cast<const float*>(smem + L.ls);
  TopBuf<float, unsigned> tb;
  tb.val[0] = reinterpret_cast<float*>(smem + L.tv0);
  tb.val[1] = reinterpret_cast<float*>(smem + L.tv1);
  tb.idx[0] = reinterpret_cast<unsigned*>(smem + L.ti0);
  tb.idx[1] = reinterpret_cast<unsigned*>(smem + L.ti1);
  tb.cnt = s_tcnt;
  float thr_hi = -pinf<float>(), thr_lo = pinf<float>();
  ThreadRed<float, unsigned> tr;
  tr.init();
  const M full = (N >= (int)(8 * sizeof(M))) ? ~(M)0 : (((M)1 << N) - 1);
  const unsigned long long n = a.rank_end - a.rank_begin;
  const unsigned long long nch = (n + chunk - 1) / chunk;
  const unsigned long long stride = (unsigned long long)gridDim.x * RED_NT;
  const unsigned long long rounds = (nch + stride - 1) / stride;
  const int trigger = TOP_CAP - RED_NT * chunk;
  const float tau_piv = a.tau_piv, tau_tr = a.tau_tr;

  for (unsigned long long rd = 0; rd < rounds; rd++) {
    const unsigned long long ch = rd * stride + (unsigned long long)blockIdx.x * RED_NT + threadIdx.x;
    if (ch < nch) {
      const unsigned long long r0 = a.rank_begin + ch * chunk;
      const unsigned long long left = a.rank_end - r0;
      const int cnt = left < (unsigned long long)chunk ? (int)left : chunk;
      M mask = unrank_s<M>(r0, K, N, sb, K + 1);
      for (int j = 0; j < cnt; j++) {
        float lr, sp, lsum, pmin, trace;
        bool bad = false;
        nplet_reg_one<K, M>(mask, N, sR, ldr, sls, lr, sp, lsum, pmin, trace, bad);
        bad |= !(pmin >= tau_piv) | !(trace <= tau_tr);
        float v[5];
        combine5<float>(lr, sp, lsum, a.cmb, v);
        const unsigned long long r = r0 + j;
        const unsigned long long gid = a.id_base + r;
        if (!red) {
          store5<float>(a, gid, v);
        } else if (!bad) {
          const unsigned loc = (unsigned)(r - a.rank_begin);
          tr.add(v, loc, lr, sp, lsum);
          if (with_top) top_offer(tb, v[3], loc, thr_hi, thr_lo);
        }
        flag_append(a, bad, gid);
        if (j + 1 < cnt) mask = lex_succ(mask, full);
      }
      tr.flush();
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
    const unsigned long long id_off = a.id_base + a.rank_begin;
    if (with_top) {
      top_sort_cut(tb, 0, a.top_m);
      top_sort_cut(tb, 1, a.top_m);
      th = tb.cnt[0];
      tl = tb.cnt[1];
      top_write(tb, a.top_m, id_off, a.part_top + (size_t)blockIdx.x * 2 * a.top_m);
    }
    block_write_part<float, unsigned>(tr, 0u, id_off, sc, a.part + blockIdx.x, th, tl);
  }
}

template <int K, typename M>
static cudaError_t launch_reg_t(const NpletArgs& a, const Shape& sh, int num_sms, cudaStream_t s,
                                int* grid_out, int max_blocks) {
  const bool red = a.mode == 1;
  const SmemLayout L = smem_layout(a.N, K, row_stride(a.N), sizeof(float), sizeof(unsigned),
                                   red && a.top_m > 0);
  void (*fn)(const NpletArgs, const int) = k_nplet_reg<K, M>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, RED_NT, L.total);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  if (sh.blocks_per_sm > 0 && sh.blocks_per_sm < occ) occ = sh.blocks_per_sm;
  int chunk = sh.chunk > 0 ? sh.chunk : 8;
  if (chunk > 8) chunk = 8;
  long long grid = (long long)num_sms * occ;
  const unsigned long long n = a.rank_end - a.rank_begin;
  const long long need = (long long)((n + (unsigned long long)RED_NT * chunk - 1) /
                                     ((unsigned long long)RED_NT * chunk));
  if (need < grid) grid = need > 0 ? need : 1;
  if (grid > max_blocks) grid = max_blocks;
  fn<<<(unsigned)grid, RED_NT, L.total, s>>>(a, chunk);
  if (grid_out) *grid_out = (int)grid;
  return cudaGetLastError();
}

template <int K>
cudaError_t launch_reg_k(const NpletArgs& a, const Shape& sh, int num_sms, cudaStream_t s,
                                int* grid_out, int max_blocks) {
  if (a.N <= 32) return launch_reg_t<K, unsigned>(a, sh, num_sms, s, grid_out, max_blocks);
  return launch_reg_t<K, unsigned long long>(a, sh, num_sms, s, grid_out, max_blocks);
}

}  // namespace thoi
