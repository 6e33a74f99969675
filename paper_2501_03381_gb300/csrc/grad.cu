// Adjoint of L = sum over nplets of one measure with respect to the
// covariance.  The paper evaluates the measures only; gradients of O are
// named as future work (Discussion).  Per nplet, with P = R_S^-1 and
// p_j = P_jj on the correlation submatrix R_S (derivatives of eq.
// gaussian_differential_entropy, d log det R = R^-1, d (R^-1)_jj =
// -(P dR P)_jj), the contribution in correlation coordinates is
//   H: 1/2 P      TC: 1/2 (I - P)      DTC: 1/2 (P - Q)
//   O: 1/2 (I - 2P + Q)                S: 1/2 (I - Q),   Q = P diag(1/p) P,
// and the gradient with respect to Sigma is G_ab / sqrt(Sigma_aa Sigma_bb).
#include <type_traits>

#include "nplet_common.cuh"

namespace thoi {

#define IXG(i, j) ((i) * ((i) + 1) / 2 + (j))
constexpr int GRAD_FLUSH = 8;  // rounds between flushes of the shared accumulator

template <typename V>
__device__ __forceinline__ V grad_entry(int measure, int a, int b, const V* P, const V* Q, int k) {
  const V pab = P[a * k + b], qab = Q[a * k + b];
  const V id = a == b ? (V)1 : (V)0;
  switch (measure) {
    case THOI_H: return (V)0.5 * pab;
    case THOI_TC: return (V)0.5 * (id - pab);
    case THOI_DTC: return (V)0.5 * (pab - qab);
    case THOI_O: return (V)0.5 * (id - (V)2 * pab + qab);
    default: return (V)0.5 * (id - qab);
  }
}

// FP32 pass over a dense rank range (flagged nplets appended to the re-factor
// list) or FP64 pass over that list.
template <typename V, int KMAX, bool LIST, typename M>
__global__ void __launch_bounds__(RED_NT) k_grad(const NpletArgs a, const int measure,
                                                 double* __restrict__ Gpart) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_stop;
  constexpr bool FP32_PATH = !LIST;
  const int N = a.N, k = a.k, ldr = row_stride(N);
  const SmemLayout L = smem_layout(N, k, ldr, sizeof(V), sizeof(unsigned), 0);
  float* Gs = reinterpret_cast<float*>(smem + L.total);  // N*N FP32 accumulator (FP32 pass)
  if (threadIdx.x == 0) s_stop = 0;
  if (FP32_PATH)
    for (int q = threadIdx.x; q < N * N; q += RED_NT) Gs[q] = 0.f;
  load_tables<V>(a, smem, L, FP32_PATH ? (const V*)a.R32 : (const V*)a.R64);
  const unsigned long long* sb = reinterpret_cast<const unsigned long long*>(smem + L.binom);
  const V* sR = reinterpret_cast<const V*>(smem + L.R);
  double* Gb = Gpart + (size_t)blockIdx.x * N * N;
  V A[KMAX * (KMAX + 1) / 2];
  V P[KMAX * KMAX];
  V Q[KMAX * KMAX];
  int c[KMAX];
  unsigned long long n;
  if (LIST) {
    const unsigned long long cnt = *a.flag_count;
    n = cnt < a.flag_cap ? cnt : a.flag_cap;
  } else {
    n = a.rank_end - a.rank_begin;
  }
  const unsigned long long stride = (unsigned long long)gridDim.x * RED_NT;
  const unsigned long long rounds = (n + stride - 1) / stride;
  for (unsigned long long rd = 0; rd < rounds; rd++) {
    const unsigned long long e = rd * stride + (unsigned long long)blockIdx.x * RED_NT + threadIdx.x;
    if (e < n) {
      unsigned long long r, gid;
      if (LIST) { gid = a.flag_ids[e]; r = gid - a.id_base; }
      else { r = a.rank_begin + e; gid = a.id_base + r; }
      M m = unrank_s<M>(r, k, N, sb, k + 1);
      for (int i = 0; i < k; i++) {
        const int hb = hibit(m);
        m ^= (M)1 << hb;
        c[i] = N - 1 - hb;
      }
      for (int i = 0; i < k; i++)
        for (int j = 0; j <= i; j++) A[IXG(i, j)] = sR[c[i] * ldr + c[j]];
      // Cholesky, smallest pivot, W = L^-1 (in place), P = W^T W
      bool bad = false;
      V pmin = pinf<V>();
      for (int p = 0; p < k; p++) {
        const V d = A[IXG(p, p)];
        pmin = d < pmin ? d : pmin;
        bad |= !pivot_ok(d);
        const V inv = (V)1 / sqrt(d);
        A[IXG(p, p)] = inv;
        for (int i = p + 1; i < k; i++) A[IXG(i, p)] *= inv;
        for (int i = p + 1; i < k; i++) {
          const V lip = A[IXG(i, p)];
          for (int j = p + 1; j <= i; j++) A[IXG(i, j)] = fma(-lip, A[IXG(j, p)], A[IXG(i, j)]);
        }
      }
      for (int j = 0; j < k; j++) {
        const V wjj = A[IXG(j, j)];
        for (int i = j + 1; i < k; i++) {
          V s = A[IXG(i, j)] * wjj;
          for (int q = j + 1; q < i; q++) s = fma(A[IXG(i, q)], A[IXG(q, j)], s);
          A[IXG(i, j)] = -A[IXG(i, i)] * s;
        }
      }
      V trace = 0;
      for (int x = 0; x < k; x++)
        for (int y = 0; y <= x; y++) {
          V s = 0;
          for (int i = x; i < k; i++) s = fma(A[IXG(i, x)], A[IXG(i, y)], s);
          P[x * k + y] = s;
          P[y * k + x] = s;
          if (x == y) trace += s;
        }
      if (FP32_PATH) {
        bad |= !(pmin >= (V)a.tau_piv) | !(trace <= (V)a.tau_tr) | !isfinite((double)trace);
        flag_append(a, bad, gid);
      } else if (bad) {
        atomicOr(a.status, ST_NOT_PD);
      }
      if (!bad) {
        for (int x = 0; x < k; x++)
          for (int y = 0; y <= x; y++) {
            V s = 0;
            for (int j = 0; j < k; j++) s += P[x * k + j] * P[j * k + y] / P[j * k + j];
            Q[x * k + y] = s;
            Q[y * k + x] = s;
          }
        for (int x = 0; x < k; x++)
          for (int y = 0; y <= x; y++) {
            const V g = grad_entry<V>(measure, x, y, P, Q, k);
            // lower triangle only (c ascending, so c[x] >= c[y]); the
            // finishing kernel mirrors it
            if (FP32_PATH) atomicAdd(&Gs[c[x] * N + c[y]], (float)g);
            else atomicAdd(&Gb[c[x] * N + c[y]], (double)g);
          }
      }
    }
    if (threadIdx.x == 0 && a.cancel && *(volatile const int*)a.cancel) s_stop = 1;
    if (FP32_PATH && ((rd + 1) % GRAD_FLUSH == 0 || rd + 1 == rounds)) {
      __syncthreads();
      for (int q = threadIdx.x; q < N * N; q += RED_NT) {
        Gb[q] += (double)Gs[q];
        Gs[q] = 0.f;
      }
    }
    __syncthreads();
    if (s_stop) {
      if (threadIdx.x == 0) atomicOr(a.status, ST_CANCELLED);
      if (FP32_PATH)
        for (int q = threadIdx.x; q < N * N; q += RED_NT) Gb[q] += (double)Gs[q];
      break;
    }
  }
}

// Sum the per-block partials (lower triangle) in block order, mirror, and
// scale to Sigma coordinates.
__global__ void k_grad_finish(const double* __restrict__ Gpart, int nblk, const double* __restrict__ sig64,
                              int N, float* __restrict__ out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * N) return;
  const int x = idx / N, y = idx % N;
  const int lo = (x > y ? x : y) * N + (x > y ? y : x);
  double s = 0;
  for (int b = 0; b < nblk; b++) s += Gpart[(size_t)b * N * N + lo];
  out[idx] = (float)(s / sqrt(sig64[x * N + x] * sig64[y * N + y]));
}

// Register-resident FP32 pass for small orders (compile-time K): the k x k
// correlation submatrix, its factor, P = R_S^-1 and Q = P diag(1/p) P live in
// registers; consecutive ranks per thread (one unrank, then the lexicographic
// successor).  Contributions go to the lower triangle of the block's shared
// FP32 accumulator, flushed into the FP64 per-block partial every round of
// GRAD_CHUNK nplets per thread.
constexpr int GRAD_CHUNK = 8;

template <int K>
__device__ __forceinline__ float grad_entry_reg(int measure, bool diag, float pab, float qab) {
  const float id = diag ? 1.f : 0.f;
  switch (measure) {
    case THOI_H: return 0.5f * pab;
    case THOI_TC: return 0.5f * (id - pab);
    case THOI_DTC: return 0.5f * (pab - qab);
    case THOI_O: return 0.5f * (id - 2.f * pab + qab);
    default: return 0.5f * (id - qab);
  }
}

template <int K, typename M>
__global__ void __launch_bounds__(RED_NT) k_grad_reg(const NpletArgs a, const int measure,
                                                     double* __restrict__ Gpart) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_stop;
  const int N = a.N, ldr = row_stride(N);
  const SmemLayout L = smem_layout(N, K, ldr, sizeof(float), sizeof(unsigned), 0);
  float* Gs = reinterpret_cast<float*>(smem + L.total);
  if (threadIdx.x == 0) s_stop = 0;
  for (int q = threadIdx.x; q < N * N; q += RED_NT) Gs[q] = 0.f;
  load_tables<float>(a, smem, L, a.R32);
  const unsigned long long* sb = reinterpret_cast<const unsigned long long*>(smem + L.binom);
  const float* sR = reinterpret_cast<const float*>(smem + L.R);
  double* Gb = Gpart + (size_t)blockIdx.x * N * N;
  const M full = (N >= (int)(8 * sizeof(M))) ? ~(M)0 : (((M)1 << N) - 1);
  const unsigned long long n = a.rank_end - a.rank_begin;
  const unsigned long long nch = (n + GRAD_CHUNK - 1) / GRAD_CHUNK;
  const unsigned long long stride = (unsigned long long)gridDim.x * RED_NT;
  const unsigned long long rounds = (nch + stride - 1) / stride;
  const float tau_piv = a.tau_piv, tau_tr = a.tau_tr;
  for (unsigned long long rd = 0; rd < rounds; rd++) {
    const unsigned long long ch = rd * stride + (unsigned long long)blockIdx.x * RED_NT + threadIdx.x;
    if (ch < nch) {
      const unsigned long long r0 = a.rank_begin + ch * GRAD_CHUNK;
      const unsigned long long left = a.rank_end - r0;
      const int cnt = left < (unsigned long long)GRAD_CHUNK ? (int)left : GRAD_CHUNK;
      M mask = unrank_s<M>(r0, K, N, sb, K + 1);
      // Consecutive ranks usually share their first K-1 variables: the
      // contributions among those (the pairs x, y < K-1) are summed in
      // registers while the prefix stays the same and added to the shared
      // accumulator when it changes.  Neighbouring lanes share prefixes too,
      // so per-nplet atomics on those pairs would serialise on one address.
      constexpr int KP = K > 1 ? K - 1 : 1;
      float Gacc[KP][KP];
      int accc[KP];
      M accp = 0;
      bool has_acc = false;
      auto flush_acc = [&]() {
#pragma unroll
        for (int x = 0; x < K - 1; x++)
#pragma unroll
          for (int y = 0; y <= x; y++) atomicAdd(&Gs[accc[x] * N + accc[y]], Gacc[x][y]);
      };
      for (int jn = 0; jn < cnt; jn++) {
        int c[K];
        {
          M m = mask;
#pragma unroll
          for (int i = 0; i < K; i++) {
            const int hb = hibit(m);
            m ^= (M)1 << hb;
            c[i] = N - 1 - hb;
          }
        }
        // Cholesky R_S = L L^T in place (1/L_pp on the diagonal)
        float A[K][K];
#pragma unroll
        for (int i = 0; i < K; i++) {
          const float* row = sR + c[i] * ldr;
#pragma unroll
          for (int j = 0; j <= i; j++) A[i][j] = row[c[j]];
        }
        float pmin = pinf<float>();
        bool bad = false;
#pragma unroll
        for (int p = 0; p < K; p++) {
          const float d = A[p][p];
          pmin = fminf(pmin, d);
          bad |= !(d > 0.f);
          const float inv = rsqrtf(d);
          A[p][p] = inv;
#pragma unroll
          for (int i = p + 1; i < K; i++) A[i][p] *= inv;
#pragma unroll
          for (int i = p + 1; i < K; i++)
#pragma unroll
            for (int j = p + 1; j <= i; j++) A[i][j] = fmaf(-A[i][p], A[j][p], A[i][j]);
        }
        // W = L^-1 in place (lower)
#pragma unroll
        for (int j = 0; j < K; j++) {
          const float wjj = A[j][j];
#pragma unroll
          for (int i = j + 1; i < K; i++) {
            float s2 = A[i][j] * wjj;
#pragma unroll
            for (int q = j + 1; q < i; q++) s2 = fmaf(A[i][q], A[q][j], s2);
            A[i][j] = -A[i][i] * s2;
          }
        }
        // P = W^T W (lower half, x >= y), p = diag(P)
        float Pm[K][K];
        float trace = 0.f;
#pragma unroll
        for (int x = 0; x < K; x++)
#pragma unroll
          for (int y = 0; y <= x; y++) {
            float s2 = 0.f;
#pragma unroll
            for (int i = x; i < K; i++) s2 = fmaf(A[i][x], A[i][y], s2);
            Pm[x][y] = s2;
            if (x == y) trace += s2;
          }
        bad |= !(pmin >= tau_piv) | !(trace <= tau_tr);
        const unsigned long long gid = a.id_base + r0 + jn;
        flag_append(a, bad, gid);
        if (!bad) {
          float dinv[K];
#pragma unroll
          for (int j = 0; j < K; j++) dinv[j] = 1.f / Pm[j][j];
          const M pmask = mask & (mask - 1);  // the nplet without its largest variable
          if (has_acc && pmask != accp) {
            flush_acc();
            has_acc = false;
          }
          if (!has_acc) {
#pragma unroll
            for (int x = 0; x < K - 1; x++) {
              accc[x] = c[x];
#pragma unroll
              for (int y = 0; y <= x; y++) Gacc[x][y] = 0.f;
            }
            accp = pmask;
            has_acc = true;
          }
#pragma unroll
          for (int x = 0; x < K; x++)
#pragma unroll
            for (int y = 0; y <= x; y++) {
              float qxy = 0.f;
              if (measure == THOI_DTC || measure == THOI_O || measure == THOI_S) {
#pragma unroll
                for (int j = 0; j < K; j++) {
                  const float pxj = j <= x ? Pm[x][j] : Pm[j][x];
                  const float pjy = j <= y ? Pm[y][j] : Pm[j][y];
                  qxy = fmaf(pxj * dinv[j], pjy, qxy);
                }
              }
              const float g = grad_entry_reg<K>(measure, x == y, Pm[x][y], qxy);
              if (x < K - 1) Gacc[x][y] += g;
              else atomicAdd(&Gs[c[x] * N + c[y]], g);
            }
        }
        if (jn + 1 < cnt) mask = lex_succ(mask, full);
      }
      if (has_acc) flush_acc();
    }
    if (threadIdx.x == 0 && a.cancel && *(volatile const int*)a.cancel) s_stop = 1;
    __syncthreads();
    for (int q = threadIdx.x; q < N * N; q += RED_NT) {
      Gb[q] += (double)Gs[q];
      Gs[q] = 0.f;
    }
    __syncthreads();
    if (s_stop) {
      if (threadIdx.x == 0) atomicOr(a.status, ST_CANCELLED);
      break;
    }
  }
}

template <int K, typename M>
static cudaError_t launch_grad_reg_t(const NpletArgs& a, double* Gpart, int grid, int measure,
                                     cudaStream_t s) {
  const SmemLayout L = smem_layout(a.N, K, row_stride(a.N), sizeof(float), sizeof(unsigned), 0);
  const size_t sm = L.total + (size_t)a.N * a.N * sizeof(float);
  void (*fn)(const NpletArgs, const int, double*) = k_grad_reg<K, M>;
  int occ = 0;
  cudaError_t e = occupancy_cached((const void*)fn, RED_NT, sm, &occ);
  if (e != cudaSuccess) return e;
  fn<<<grid, RED_NT, sm, s>>>(a, measure, Gpart);
  return cudaGetLastError();
}

template <int K>
static cudaError_t launch_grad_reg_k(const NpletArgs& a, double* Gpart, int grid, int measure,
                                     cudaStream_t s) {
  if (a.N > 32) return launch_grad_reg_t<K, unsigned long long>(a, Gpart, grid, measure, s);
  return launch_grad_reg_t<K, unsigned>(a, Gpart, grid, measure, s);
}

template <typename V, int KMAX, bool LIST>
static cudaError_t launch_grad_t(const NpletArgs& a, double* Gpart, int grid, int measure,
                                 cudaStream_t s) {
  const SmemLayout L = smem_layout(a.N, a.k, row_stride(a.N), sizeof(V), sizeof(unsigned), 0);
  const size_t sm = L.total + (LIST ? 0 : (size_t)a.N * a.N * sizeof(float));
  void (*fn)(const NpletArgs, const int, double*);
  if (a.N > 32) fn = k_grad<V, KMAX, LIST, unsigned long long>;
  else fn = k_grad<V, KMAX, LIST, unsigned>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  fn<<<grid, RED_NT, sm, s>>>(a, measure, Gpart);
  return cudaGetLastError();
}

// grid: number of blocks (<= the Gpart regions allocated).
cudaError_t launch_grad_pass(const NpletArgs& a, double* Gpart, int grid, int measure, bool list,
                             cudaStream_t s) {
  if (!list) {
    switch (a.k) {
      case 1: return launch_grad_reg_k<1>(a, Gpart, grid, measure, s);
      case 2: return launch_grad_reg_k<2>(a, Gpart, grid, measure, s);
      case 3: return launch_grad_reg_k<3>(a, Gpart, grid, measure, s);
      case 4: return launch_grad_reg_k<4>(a, Gpart, grid, measure, s);
      case 5: return launch_grad_reg_k<5>(a, Gpart, grid, measure, s);
      case 6: return launch_grad_reg_k<6>(a, Gpart, grid, measure, s);
      case 7: return launch_grad_reg_k<7>(a, Gpart, grid, measure, s);
      case 8: return launch_grad_reg_k<8>(a, Gpart, grid, measure, s);
      default: break;
    }
  }
  const int kb = a.k <= 8 ? 8 : (a.k <= 16 ? 16 : 32);
  if (list) {
    if (kb == 8) return launch_grad_t<double, 8, true>(a, Gpart, grid, measure, s);
    if (kb == 16) return launch_grad_t<double, 16, true>(a, Gpart, grid, measure, s);
    return launch_grad_t<double, 32, true>(a, Gpart, grid, measure, s);
  }
  if (kb == 8) return launch_grad_t<float, 8, false>(a, Gpart, grid, measure, s);
  if (kb == 16) return launch_grad_t<float, 16, false>(a, Gpart, grid, measure, s);
  return launch_grad_t<float, 32, false>(a, Gpart, grid, measure, s);
}

cudaError_t launch_grad_finish(const double* Gpart, int nblk, const double* sig64, int N, float* out,
                               cudaStream_t s) {
  k_grad_finish<<<(N * N + 255) / 256, 256, 0, s>>>(Gpart, nblk, sig64, N, out);
  return cudaGetLastError();
}

}  // namespace thoi
