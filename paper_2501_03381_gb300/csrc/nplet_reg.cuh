// Register-resident FP32 nplet kernel (templates), one template instance per order
// k <= 24: each thread owns one nplet at a time, its k x k correlation
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
// so their shared-memory gathers mostly hit the same words.  Output: mode 0
// writes the five measures per nplet, mode 2 the three basis values that the
// streaming reduction consumes, mode 3 reduces in place (fused records);
// flagged nplets go to the FP64 re-factor list.
// Minimum resident blocks per SM, picked per order by timing: orders up to
// 16 are held to three blocks (at most 168 registers a thread), 18..20 to two;
// order 17 keeps the allocation the compiler picks on its own (three blocks
// spill there, two are slower than one), and so do 21..24, which reach the
// 255-register limit and spill a little.
template <int K>
struct RegBlocks {
  static constexpr int value = K <= 16 ? 3 : ((K == 17 || K > 20) ? 1 : 2);
};

// Per-nplet output (mode 0) goes through shared memory: the 32 lanes of a
// warp hold 32 consecutive chunks, i.e. 32 * chunk consecutive ranks, so the
// warp stages their values and writes each measure's run with consecutive
// lanes on consecutive addresses (a direct store from each lane's own chunk
// would touch 32 sectors per instruction).
constexpr int REG_STAGE = 5 * 32 * 8;  // floats staged per warp (five measures, chunk <= 8)
constexpr size_t REG_STAGE_BYTES = (size_t)(RED_NT / 32) * REG_STAGE * sizeof(float);

template <int K, typename M>
__global__ void __launch_bounds__(RED_NT, RegBlocks<K>::value) k_nplet_reg(const NpletArgs a,
                                                                          const int chunk) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = a.N, ldr = row_stride(N);
  const SmemLayout L = smem_layout(N, K, ldr, sizeof(float), sizeof(unsigned), 0);
  load_tables<float>(a, smem, L, a.R32);
  const unsigned long long* sb = reinterpret_cast<const unsigned long long*>(smem + L.binom);
  const float* sR = reinterpret_cast<const float*>(smem + L.R);
  const float* sls = reinterpret_cast<const float*>(smem + L.ls);
  const bool basis = a.mode == 2;
  const bool fused = a.mode == 3;
  const bool stage = a.mode == 0;
  const float* sthr = reinterpret_cast<const float*>(smem + L.thr);
  const int lane = threadIdx.x & 31;
  float* sbuf = reinterpret_cast<float*>(smem + L.total) + (threadIdx.x >> 5) * REG_STAGE;
  FusedAcc acc;
  acc.init();
  const M full = (N >= (int)(8 * sizeof(M))) ? ~(M)0 : (((M)1 << N) - 1);
  const unsigned long long n = a.rank_end - a.rank_begin;
  const unsigned long long nch = (n + chunk - 1) / chunk;
  const unsigned long long stride = (unsigned long long)gridDim.x * RED_NT;
  const float tau_piv = a.tau_piv, tau_tr = a.tau_tr;
  const CombineV<float> cmbv(a.cmb);

  if (a.mode == 4) {
    // sample bounds of fused records: `chunk` samples per thread, sample i of
    // S taken by block i % grid, every sample unranked on its own
    const unsigned long long S0 = (unsigned long long)gridDim.x * RED_NT * (unsigned)chunk;
    const unsigned long long S = n < S0 ? n : S0;
    float mn[5], mx[5];
#pragma unroll
    for (int m = 0; m < 5; m++) {
      mn[m] = pinf<float>();
      mx[m] = -pinf<float>();
    }
    unsigned valid = 0;
    for (int e = 0; e < chunk; e++) {
      const unsigned long long i =
          ((unsigned long long)threadIdx.x * chunk + e) * gridDim.x + blockIdx.x;
      if (i >= S) continue;
      const M mask = unrank_s<M>(sample_rank(a, i, S), K, N, sb, K + 1);
      float lr, sp, lsum, pmin, trace;
      bool bad = false;
      nplet_reg_one<K, M>(mask, N, sR, ldr, sls, lr, sp, lsum, pmin, trace, bad);
      bad |= !(pmin >= tau_piv) | !(trace <= tau_tr);
      if (bad) continue;
      float v[5];
      combine5<float>(lr, sp, lsum, cmbv, v);
#pragma unroll
      for (int m = 0; m < 5; m++) {
        mn[m] = fminf(mn[m], v[m]);
        mx[m] = fmaxf(mx[m], v[m]);
      }
      valid++;
    }
    sample_block_keys(a, mn, mx, valid);
    return;
  }

  // whole warps step together (lane l takes chunk chw + l), so that the
  // staged output of a warp is one contiguous run of ranks
  for (unsigned long long chw = (unsigned long long)blockIdx.x * RED_NT + (threadIdx.x & ~31u);
       chw < nch; chw += stride) {
    // the cancel flag lives in host memory: read it once every 64 rounds
    if (((chw / stride) & 63) == 0 && a.cancel && *(volatile const int*)a.cancel) {
      if (lane == 0) atomicOr(a.status, ST_CANCELLED);
      break;
    }
    const unsigned long long ch = chw + lane;
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
        const unsigned long long gid = a.id_base + r0 + j;
        if (fused) {
          fused_emit(a, acc, sthr, cmbv, gid, lr, sp, lsum, bad);
        } else {
          if (basis) {
            store_basis(a, gid, lr, sp, lsum, bad);
          } else {
            float v[5];
            combine5<float>(lr, sp, lsum, cmbv, v);
            const int e = lane * chunk + j;
#pragma unroll
            for (int m = 0; m < 5; m++) sbuf[m * 32 * 8 + e] = v[m];
          }
          flag_append(a, bad, gid);
        }
        if (j + 1 < cnt) mask = lex_succ(mask, full);
      }
    }
    if (stage) {
      __syncwarp();
      const unsigned long long wr0 = a.rank_begin + chw * chunk;
      const unsigned long long wleft = a.rank_end - wr0;
      const int wn = wleft < (unsigned long long)(32 * chunk) ? (int)wleft : 32 * chunk;
      const unsigned long long o0 = a.id_base + wr0 - a.out_first;
      const int m0 = a.out_sel > 0 ? a.out_sel - 1 : 0, m1 = a.out_sel > 0 ? a.out_sel : 5;
      for (int m = m0; m < m1; m++) {
        const unsigned long long row = a.out_sel > 0 ? 0ull : (unsigned long long)m * a.out_n;
        if (a.out_f64) {
          double* O = reinterpret_cast<double*>(a.out) + row + o0;
          for (int e = lane; e < wn; e += 32) O[e] = (double)sbuf[m * 32 * 8 + e];
        } else {
          float* O = reinterpret_cast<float*>(a.out) + row + o0;
          for (int e = lane; e < wn; e += 32) O[e] = sbuf[m * 32 * 8 + e];
        }
      }
      __syncwarp();
    }
  }
  if (fused) fused_block_end(a, acc);
}

template <int K, typename M>
static cudaError_t launch_reg_t(const NpletArgs& a, const Shape& sh, int num_sms, cudaStream_t s,
                                int* grid_out, int max_blocks) {
  const SmemLayout L = smem_layout(a.N, K, row_stride(a.N), sizeof(float), sizeof(unsigned), 0);
  const size_t smem = L.total + (a.mode == 0 ? REG_STAGE_BYTES : 0);
  void (*fn)(const NpletArgs, const int) = k_nplet_reg<K, M>;
  int occ = 0;
  cudaError_t e = occupancy_cached((const void*)fn, RED_NT, smem, &occ);
  if (e != cudaSuccess) return e;
  if (a.mode == 4) {
    // sample bounds: max(256, top_m) blocks (so that the smallest block
    // maximum has at least top_m samples at or above it), sh.chunk samples
    // per thread
    const int sgrid = a.top_m > 256 ? a.top_m : 256;
    fn<<<(unsigned)sgrid, RED_NT, smem, s>>>(a, sh.chunk > 0 ? sh.chunk : 1);
    if (grid_out) *grid_out = sgrid;
    return cudaGetLastError();
  }
  if (sh.blocks_per_sm > 0 && sh.blocks_per_sm < occ) occ = sh.blocks_per_sm;
  int chunk = sh.chunk > 0 ? sh.chunk : 8;
  if (chunk > 8) chunk = 8;
  long long grid = (long long)num_sms * occ;
  const unsigned long long n = a.rank_end - a.rank_begin;
  const long long need = (long long)((n + (unsigned long long)RED_NT * chunk - 1) /
                                     ((unsigned long long)RED_NT * chunk));
  if (need < grid) grid = need > 0 ? need : 1;
  if (grid > max_blocks) grid = max_blocks;
  fn<<<(unsigned)grid, RED_NT, smem, s>>>(a, chunk);
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
