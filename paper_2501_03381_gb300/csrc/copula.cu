// Gaussian-copula front end (Supp. eq. gaussian_copula_covariance_estimator):
// per-column ordinal rank -> u = (r+1)/(T+1) -> z = Phi^{-1}(u) -> centred
// covariance divided by T-1, in FP64 on CUDA cores and, for the FP32 path, as
// a split-BF16 tensor-core GEMM with FP32 accumulation.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace thoi {

// ---------------------------------------------------------------- K1: rank
// Ordinal rank of sample t in column j: #{s : x_s < x_t} + #{s < t : x_s == x_t}.
// Equal values keep sample order; -0.0 == +0.0 under IEEE comparison.  One
// thread per sample, the column streamed through shared memory in tiles.
constexpr int RANK_NT = 256;
constexpr int RANK_TILE = 4096;

template <typename F>
__global__ void __launch_bounds__(RANK_NT) k_rank(const F* __restrict__ X, long long T, int N,
                                                  long long ld, int* __restrict__ rank,
                                                  int* status) {
  __shared__ F tile[RANK_TILE];
  const int j = blockIdx.x;
  const long long t = (long long)blockIdx.y * RANK_NT + threadIdx.x;
  F xt = 0;
  if (t < T) {
    xt = X[t * ld + j];
    if (!isfinite((double)xt)) atomicOr(status, ST_NONFINITE);
  }
  long long cnt = 0;
  for (long long s0 = 0; s0 < T; s0 += RANK_TILE) {
    const int len = (int)min((long long)RANK_TILE, T - s0);
    __syncthreads();
    for (int q = threadIdx.x; q < len; q += RANK_NT) tile[q] = X[(s0 + q) * ld + j];
    __syncthreads();
    if (t < T) {
      for (int q = 0; q < len; q++) {
        const F xs = tile[q];
        cnt += (xs < xt) | ((xs == xt) & (s0 + q < t));
      }
    }
  }
  if (t < T) rank[t * N + j] = (int)cnt;
}

// ---------------------------------------------------------------- K2: Phi^{-1}
// ztab[r] = Phi^{-1}((r+1)/(T+1)), evaluated from the nearer tail so that the
// upper half keeps full precision: Phi^{-1}(u) = -Phi^{-1}(1-u).
__global__ void k_ztab(long long T, double* __restrict__ ztab) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= T) return;
  const double den = (double)(T + 1);
  const long long num = r + 1;
  double z;
  if (2 * num == T + 1) z = 0.0;
  else if (2 * num < T + 1) z = normcdfinv((double)num / den);
  else z = -normcdfinv((double)(T + 1 - num) / den);
  ztab[r] = z;
}

// Z (variable-major, N x T): Z[j][t] = ztab[rank[t][j]]; then the column mean.
__global__ void k_apply_z(const int* __restrict__ rank, const double* __restrict__ ztab,
                          long long T, int N, double* __restrict__ Z) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= T * N) return;
  const long long t = idx / N;
  const int j = (int)(idx % N);
  Z[(long long)j * T + t] = ztab[rank[idx]];
}

constexpr int RED_T = 256;
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0;
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)(blockDim.x >> 5); q++) s += sh[q];
  return s;  // valid in thread 0
}

__global__ void __launch_bounds__(RED_T) k_mean(const double* __restrict__ Z, long long T,
                                                double* __restrict__ mu) {
  __shared__ double sh[RED_T / 32];
  const int j = blockIdx.x;
  double s = 0;
  for (long long t = threadIdx.x; t < T; t += RED_T) s += Z[(long long)j * T + t];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) mu[j] = s / (double)T;
}

// ---------------------------------------------------------------- K3b: FP64 covariance
// Sigma_ij = sum_t (z_ti - mu_i)(z_tj - mu_j) / (T - 1); one block per (i, j <= i).
__global__ void __launch_bounds__(RED_T) k_cov64(const double* __restrict__ Z,
                                                 const double* __restrict__ mu, long long T,
                                                 int N, double* __restrict__ sig) {
  __shared__ double sh[RED_T / 32];
  int p = blockIdx.x;
  int i = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
  while ((i + 1) * (i + 2) / 2 <= p) i++;
  while (i * (i + 1) / 2 > p) i--;
  const int j = p - i * (i + 1) / 2;
  const double mi = mu[i], mj = mu[j];
  double s = 0;
  for (long long t = threadIdx.x; t < T; t += RED_T)
    s = fma(Z[(long long)i * T + t] - mi, Z[(long long)j * T + t] - mj, s);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    const double v = s / (double)(T - 1);
    sig[i * N + j] = v;
    sig[j * N + i] = v;
  }
}

// ---------------------------------------------------------------- K3: split-BF16 tensor-core covariance
// Zc = Z - mu is split into three BF16 terms hi + mid + lo (8 significant
// bits each, 24 together).  The six products whose combined weight is at
// most 2^-16 relative (hi.hi, hi.mid, mid.hi, hi.lo, lo.hi, mid.mid) are
// summed by mma.sync m16n8k16 into an FP32 accumulator that starts from zero
// for every 16-sample step; the step sums are then added in FP64.  Letting
// one FP32 tensor-core accumulator run over many steps biases the diagonal
// by about -2.4e-6 relative (the accumulator add truncates), which moves O
// by more than 1e-4 at k >= 20.
constexpr int TC_CHUNK = 256;

__global__ void k_split_bf16(const double* __restrict__ Z, const double* __restrict__ mu,
                             long long T, long long Tp, int N, int Np,
                             __nv_bfloat16* __restrict__ zh, __nv_bfloat16* __restrict__ zm,
                             __nv_bfloat16* __restrict__ zl) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)Np * Tp) return;
  const int j = (int)(idx / Tp);
  const long long t = idx % Tp;
  double v = 0.0;
  if (j < N && t < T) v = Z[(long long)j * T + t] - mu[j];
  const float vf = (float)v;
  const __nv_bfloat16 h = __float2bfloat16_rn(vf);
  const float r1 = vf - __bfloat162float(h);
  const __nv_bfloat16 m = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(m);
  const __nv_bfloat16 l = __float2bfloat16_rn(r2);
  zh[idx] = h;
  zm[idx] = m;
  zl[idx] = l;
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4],
                                         const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One warp per (16 x 8 output tile, chunk of 256 samples).  A fragment rows
// are variables i0..i0+15, B fragment columns variables j0..j0+7, K = samples.
__global__ void k_cov_tc(const __nv_bfloat16* __restrict__ zh, const __nv_bfloat16* __restrict__ zm,
                         const __nv_bfloat16* __restrict__ zl, long long Tp, int Np, int tiles_j,
                         int n_tiles, double* __restrict__ part) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int tile = warp % n_tiles;
  const int chunk = warp / n_tiles;
  const long long t_begin = (long long)chunk * TC_CHUNK;
  if (t_begin >= Tp) return;
  const int i0 = (tile / tiles_j) * 16, j0 = (tile % tiles_j) * 8;
  const int g = lane >> 2, q = lane & 3;
  double acc64[4] = {0.0, 0.0, 0.0, 0.0};
  const long long t_end = min(Tp, t_begin + TC_CHUNK);
  const __nv_bfloat16* srcs[3] = {zh, zm, zl};
  for (long long t0 = t_begin; t0 < t_end; t0 += 16) {
    unsigned a[3][4], b[3][2];
#pragma unroll
    for (int s = 0; s < 3; s++) {
      const __nv_bfloat16* Zs = srcs[s];
      const long long ra = (long long)(i0 + g) * Tp + t0 + 2 * q;
      const long long rb = (long long)(i0 + g + 8) * Tp + t0 + 2 * q;
      const long long rj = (long long)(j0 + g) * Tp + t0 + 2 * q;
      a[s][0] = *reinterpret_cast<const unsigned*>(Zs + ra);
      a[s][1] = *reinterpret_cast<const unsigned*>(Zs + rb);
      a[s][2] = *reinterpret_cast<const unsigned*>(Zs + ra + 8);
      a[s][3] = *reinterpret_cast<const unsigned*>(Zs + rb + 8);
      b[s][0] = *reinterpret_cast<const unsigned*>(Zs + rj);
      b[s][1] = *reinterpret_cast<const unsigned*>(Zs + rj + 8);
    }
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    // smallest terms first
    mma_bf16(acc, a[1], b[1]);  // mid.mid
    mma_bf16(acc, a[0], b[2]);  // hi.lo
    mma_bf16(acc, a[2], b[0]);  // lo.hi
    mma_bf16(acc, a[0], b[1]);  // hi.mid
    mma_bf16(acc, a[1], b[0]);  // mid.hi
    mma_bf16(acc, a[0], b[0]);  // hi.hi
#pragma unroll
    for (int r = 0; r < 4; r++) acc64[r] += (double)acc[r];
  }
  // C fragment: (row g, cols 2q, 2q+1) and (row g+8, same cols)
  double* P = part + (long long)chunk * Np * Np;
  P[(i0 + g) * Np + j0 + 2 * q] = acc64[0];
  P[(i0 + g) * Np + j0 + 2 * q + 1] = acc64[1];
  P[(i0 + g + 8) * Np + j0 + 2 * q] = acc64[2];
  P[(i0 + g + 8) * Np + j0 + 2 * q + 1] = acc64[3];
}

// Sum the per-chunk tiles in FP64 (fixed chunk order), scale by 1/(T-1).
__global__ void k_cov_tc_sum(const double* __restrict__ part, int n_chunks, int Np, int N,
                             long long T, double* __restrict__ sig32acc) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * N) return;
  const int i = idx / N, j = idx % N;
  double s = 0;
  for (int c = 0; c < n_chunks; c++) s += part[(long long)c * Np * Np + i * Np + j];
  sig32acc[idx] = s / (double)(T - 1);
}

// ---------------------------------------------------------------- normalisation
// R = D^-1/2 Sigma D^-1/2 (FP64 from Sigma64; FP32 from the tensor-core
// covariance, or from Sigma64 when that is the chosen source) and
// ls_i = log Sigma64_ii.  TC, DTC, O and S are invariant under per-variable
// scaling, so the nplet kernels work on R; H adds back sum_i ls_i.
__global__ void k_normalise(const double* __restrict__ sig64, const double* __restrict__ sig32acc,
                            int N, double* __restrict__ R64, float* __restrict__ R32,
                            double* __restrict__ ls, float* __restrict__ sig32_out, int* status) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * N) return;
  const int i = idx / N, j = idx % N;
  const double di = sig64[i * N + i], dj = sig64[j * N + j];
  if (!(di > 0.0) || !(dj > 0.0) || !isfinite(di) || !isfinite(dj)) {
    atomicOr(status, ST_BAD_ARG);
    return;
  }
  R64[idx] = (i == j) ? 1.0 : sig64[idx] / sqrt(di * dj);
  const double* s32 = sig32acc ? sig32acc : sig64;
  const double ei = s32[i * N + i], ej = s32[j * N + j];
  R32[idx] = (i == j) ? 1.0f : (float)(s32[idx] / sqrt(ei * ej));
  if (sig32_out) sig32_out[idx] = (float)s32[idx];
  if (i == j) ls[i] = log(di);
}

// ---------------------------------------------------------------- launchers
void copula_ws_sizes(long long T, int N, CopulaWsSizes* z) {
  z->Np = (N + 15) / 16 * 16;
  z->Tp = (T + 15) / 16 * 16;
  z->n_chunks = (int)((z->Tp + TC_CHUNK - 1) / TC_CHUNK);
}

cudaError_t launch_copula(const void* X, int dtype, long long T, int N, long long ld,
                          const CopulaWs& w, int tc_cov, int* d_status, cudaStream_t s) {
  dim3 g1(N, (unsigned)((T + RANK_NT - 1) / RANK_NT));
  if (dtype == THOI_DTYPE_F64)
    k_rank<double><<<g1, RANK_NT, 0, s>>>((const double*)X, T, N, ld, w.rank, d_status);
  else
    k_rank<float><<<g1, RANK_NT, 0, s>>>((const float*)X, T, N, ld, w.rank, d_status);
  k_ztab<<<(unsigned)((T + 255) / 256), 256, 0, s>>>(T, w.ztab);
  k_apply_z<<<(unsigned)((T * N + 255) / 256), 256, 0, s>>>(w.rank, w.ztab, T, N, w.Z);
  k_mean<<<N, RED_T, 0, s>>>(w.Z, T, w.mu);
  k_cov64<<<N * (N + 1) / 2, RED_T, 0, s>>>(w.Z, w.mu, T, N, w.sig64);
  if (tc_cov) {
    CopulaWsSizes z;
    copula_ws_sizes(T, N, &z);
    __nv_bfloat16* zh = (__nv_bfloat16*)w.zh;
    __nv_bfloat16* zm = (__nv_bfloat16*)w.zm;
    __nv_bfloat16* zl = (__nv_bfloat16*)w.zl;
    const long long nz = (long long)z.Np * z.Tp;
    k_split_bf16<<<(unsigned)((nz + 255) / 256), 256, 0, s>>>(w.Z, w.mu, T, z.Tp, N, z.Np, zh, zm,
                                                             zl);
    const int tiles_j = z.Np / 8;
    const int n_tiles = (z.Np / 16) * tiles_j;
    const long long warps = (long long)n_tiles * z.n_chunks;
    k_cov_tc<<<(unsigned)((warps + 3) / 4), 128, 0, s>>>(zh, zm, zl, z.Tp, z.Np, tiles_j, n_tiles,
                                                       w.part);
    k_cov_tc_sum<<<(N * N + 255) / 256, 256, 0, s>>>(w.part, z.n_chunks, z.Np, N, T, w.sig32acc);
  }
  return cudaGetLastError();
}

cudaError_t launch_normalise(const double* sig64, const double* sig32acc, int N, double* R64,
                             float* R32, double* ls, float* sig32_out, int* status,
                             cudaStream_t s) {
  k_normalise<<<(N * N + 255) / 256, 256, 0, s>>>(sig64, sig32acc, N, R64, R32, ls, sig32_out,
                                                  status);
  return cudaGetLastError();
}

}  // namespace thoi
