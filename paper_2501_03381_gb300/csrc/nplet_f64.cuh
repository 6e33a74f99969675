// FP64 shared-memory nplet computation (body shared by the single-order and
// the batched kernels); see nplet_f64.cu.
#pragma once
#include "nplet_common.cuh"

namespace thoi {

template <int NT, bool LIST, typename M>
__device__ void f64s_body(const NpletArgs& a, double* __restrict__ b64, unsigned long long bstride,
                          unsigned char* smem) {
  const int N = a.N, k = a.k, ldr = row_stride(N);
  const SmemLayout L = smem_layout(N, k, ldr, sizeof(double), 8, 0);
  load_tables<double>(a, smem, L, a.R64);
  const unsigned long long* sb = reinterpret_cast<const unsigned long long*>(smem + L.binom);
  const double* sR = reinterpret_cast<const double*>(smem + L.R);
  const double* sls = reinterpret_cast<const double*>(smem + L.ls);
  double* A = reinterpret_cast<double*>(smem + L.total) + threadIdx.x;
#define AE(i, j) A[(size_t)((((i) * ((i) + 1)) >> 1) + (j)) * NT]
  const CombineV<double> cmbv(a.cmb);
  unsigned long long n;
  if (LIST) {
    const unsigned long long c = *a.flag_count;
    n = c < a.flag_cap ? c : a.flag_cap;
  } else {
    n = a.rank_end - a.rank_begin;
  }
  int c[THOI_MAX_N];
  for (unsigned long long e = (unsigned long long)blockIdx.x * NT + threadIdx.x; e < n;
       e += (unsigned long long)gridDim.x * NT) {
    unsigned long long r, gid;
    if (LIST) {
      gid = a.flag_ids[e];
      r = gid - a.id_base;
    } else {
      r = a.rank_begin + e;
      gid = a.id_base + r;
    }
    M m = unrank_s<M>(r, k, N, sb, k + 1);
    for (int i = 0; i < k; i++) {
      const int hb = hibit(m);
      m ^= (M)1 << hb;
      c[i] = N - 1 - hb;
    }
    double lsum = 0.0;
    for (int i = 0; i < k; i++) {
      const double* row = sR + c[i] * ldr;
      lsum += sls[c[i]];
      for (int j = 0; j <= i; j++) AE(i, j) = row[c[j]];
    }
    // LDL^T in place (rows updated from the bottom so column p is read before
    // it is scaled)
    double P1 = 1.0, P2 = 1.0;
    int E1 = 0, E2 = 0;
    bool bad = false;
    for (int p = 0; p < k; p++) {
      const double d = AE(p, p);
      bad |= !pivot_ok(d);
      P1 *= d;
      if ((p & 7) == 7 || p == k - 1) renorm(P1, E1, bad);
      const double rd = 1.0 / d;
      AE(p, p) = rd;
      for (int i = k - 1; i > p; i--) {
        const double u = AE(i, p) * rd;
        for (int j = p + 1; j <= i; j++) AE(i, j) = fma(-u, AE(j, p), AE(i, j));
        AE(i, p) = u;
      }
    }
    // unit-lower inverse, column by column, and the inverse diagonal
    for (int j = 0; j < k; j++) {
      double pj = AE(j, j);
      for (int i = j + 1; i < k; i++) {
        double s = AE(i, j);
        for (int q = j + 1; q < i; q++) s = fma(-AE(i, q), AE(q, j), s);
        AE(i, j) = s;
        pj = fma(s * AE(i, i), s, pj);
      }
      P2 *= pj;
      if ((j & 7) == 7 || j == k - 1) renorm(P2, E2, bad);
    }
    const double lr = log_of(P1, E1), sp = log_of(P2, E2);
    if (bad) atomicOr(a.status, ST_NOT_PD);
    if (a.mode == 0) {
      double v[5];
      combine5<double>(lr, sp, lsum, cmbv, v);
      if (bad)
        for (int q = 0; q < 5; q++) v[q] = __longlong_as_double(0x7ff8000000000000ll);
      store5<double>(a, gid, v);
    } else {
      b64[e] = bad ? __longlong_as_double(0x7ff8000000000000ll) : lr;
      b64[bstride + e] = sp;
      b64[2 * bstride + e] = lsum;
    }
  }
#undef AE
}

}  // namespace thoi

namespace thoi {

// The factorisation steps of a group of G lanes on the k x k lower triangle
// A (packed by rows, row i owned by lane i mod G; the lanes of gmask meet at
// warp barriers): LDL^T (1/D_p left on the diagonal), V = L^-1 in place, and
// the inverse diagonal p_j.  Lane 0 returns the product of the 1/D_p in
// (P1, E1) and every lane the product of the p_j in (P2, E2); bad is set on
// lane 0 for a pivot that is not positive and finite, and on every lane for
// an overflowing p_j product.
template <int G>
__device__ __forceinline__ void f64g_factor(double* __restrict__ A, const int k, const int g,
                                            const unsigned gmask, double& P1, int& E1,
                                            double& P2, int& E2, bool& bad) {
#define AG(i, j) A[((((i) * ((i) + 1)) >> 1) + (j))]
  // LDL^T
  for (int p = 0; p < k; p++) {
    // the owner of row p divides once and publishes 1/D_p on the diagonal
    // (an FP64 division is a long sequence on the narrow FP64 pipe); lane
    // 0 keeps the product of the 1/D_p, so log det R_S = -log(product)
    if (g == p % G) AG(p, p) = 1.0 / AG(p, p);
    __syncwarp(gmask);
    const double rd = AG(p, p);
    if (g == 0) {
      bad |= !rcp_pivot_ok(rd);  // D_p <= 2^-45, zero, or not finite
      P1 *= rd;
      if ((p & 7) == 7 || p == k - 1) renorm(P1, E1, bad);
    }
    const int i0 = p + 1 + ((g - (p + 1) % G) + G) % G;  // first owned row > p
    // the multipliers of the owned rows are kept, then written over column p
    // once every row has read it
    double us[32 / G + 1];
#pragma unroll
    for (int t = 0; t < 32 / G + 1; t++) {
      const int i = i0 + t * G;
      if (i < k) {
        const double u = AG(i, p) * rd;
        for (int j = p + 1; j <= i; j++) AG(i, j) = fma(-u, AG(j, p), AG(i, j));
        us[t] = u;
      }
    }
    __syncwarp(gmask);
#pragma unroll
    for (int t = 0; t < 32 / G + 1; t++) {
      const int i = i0 + t * G;
      if (i < k) AG(i, p) = us[t];
    }
    __syncwarp(gmask);
  }
  // V = L^-1 in place
  for (int mm = 0; mm + 1 < k; mm++) {
    const int i0 = mm + 1 + ((g - (mm + 1) % G) + G) % G;
    for (int i = i0; i < k; i += G) {
      const double l = AG(i, mm);
      for (int c = 0; c < mm; c++) AG(i, c) = fma(-l, AG(mm, c), AG(i, c));
      AG(i, mm) = -l;
    }
    __syncwarp(gmask);
  }
  // inverse diagonal, product of the p_j across the group
  bool bad2 = false;
  for (int j = g; j < k; j += G) {
    double pj = AG(j, j);
    for (int i = j + 1; i < k; i++) {
      const double v = AG(i, j);
      pj = fma(v * AG(i, i), v, pj);
    }
    P2 *= pj;
    renorm(P2, E2, bad2);
  }
#pragma unroll
  for (int o = 1; o < G; o <<= 1) {
    const double q = __shfl_xor_sync(gmask, P2, o);
    const int eq = __shfl_xor_sync(gmask, E2, o);
    P2 *= q;
    E2 += eq;
    renorm(P2, E2, bad2);
  }
  bad |= __any_sync(gmask, bad2);
#undef AG
}

// FP64 nplet computation with G lanes per nplet: the group's k x k matrix
// (lower triangle) and index list live in shared memory, rows are owned
// cyclically (row i by lane i mod G), and the lanes meet at a warp barrier
// after every elimination step.  With one nplet per thread a block of
// large-order matrices fills the shared memory with one or two warps, which
// leaves schedulers without FP64 work; sharing a matrix among G lanes gives
// G times as many warps for the same shared memory.
//
//   LDL^T, right-looking: step p updates the owned rows i > p with the
//     unscaled column p, then (after a barrier) scales the owned column
//     entries to L^_ip and stores 1/D_p on the diagonal.
//   V = L^-1 (unit lower), right-looking and in place: step m subtracts
//     L^_im times the finished row m from every owned row i > m; entry
//     (i, m) becomes -L^_im, and row i is final after step i - 1.
//   p_j = 1/D_j + sum_{i>j} V_ij^2 / D_i, column j by lane j mod G; the
//     product of the p_j and the sum of log Sigma_ii are combined across the
//     group with shuffles.
template <int NT, int G, bool LIST, typename M>
__device__ void f64g_body(const NpletArgs& a, double* __restrict__ b64, unsigned long long bstride,
                          unsigned char* smem) {
  constexpr int GPB = NT / G;  // nplets per block at a time
  const int N = a.N, k = a.k, ldr = row_stride(N);
  const SmemLayout L = smem_layout(N, k, ldr, sizeof(double), 8, 0);
  load_tables<double>(a, smem, L, a.R64);
  const unsigned long long* sb = reinterpret_cast<const unsigned long long*>(smem + L.binom);
  const double* sR = reinterpret_cast<const double*>(smem + L.R);
  const double* sls = reinterpret_cast<const double*>(smem + L.ls);
  const int tri = k * (k + 1) / 2;
  const int lane = threadIdx.x & 31, g = lane % G, grp = threadIdx.x / G;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane - g));
  double* A = reinterpret_cast<double*>(smem + L.total) + (size_t)grp * tri;
  int* C = reinterpret_cast<int*>(smem + L.total + (size_t)GPB * tri * sizeof(double)) + grp * k;
#define AG(i, j) A[((((i) * ((i) + 1)) >> 1) + (j))]
  const CombineV<double> cmbv(a.cmb);
  unsigned long long n;
  if (LIST) {
    const unsigned long long c = *a.flag_count;
    n = c < a.flag_cap ? c : a.flag_cap;
  } else {
    n = a.rank_end - a.rank_begin;
  }
  for (unsigned long long e = (unsigned long long)blockIdx.x * GPB + grp; e < n;
       e += (unsigned long long)gridDim.x * GPB) {
    unsigned long long r, gid;
    if (LIST) {
      gid = a.flag_ids[e];
      r = gid - a.id_base;
    } else {
      r = a.rank_begin + e;
      gid = a.id_base + r;
    }
    // indices (every lane decodes, lane g stores the positions it owns)
    M m = unrank_s<M>(r, k, N, sb, k + 1);
    for (int q = 0; q < k; q++) {
      const int hb = hibit(m);
      m ^= (M)1 << hb;
      if (q % G == g) C[q] = N - 1 - hb;
    }
    __syncwarp(gmask);
    double lsum = 0.0;
    for (int i = g; i < k; i += G) {
      const int ci = C[i];
      const double* row = sR + ci * ldr;
      lsum += sls[ci];
      for (int j = 0; j <= i; j++) AG(i, j) = row[C[j]];
    }
#pragma unroll
    for (int o = 1; o < G; o <<= 1) lsum += __shfl_xor_sync(gmask, lsum, o);
    __syncwarp(gmask);
    double P1 = 1.0, P2 = 1.0;
    int E1 = 0, E2 = 0;
    bool bad = false;
    f64g_factor<G>(A, k, g, gmask, P1, E1, P2, E2, bad);
    if (g == 0) {
      const double lr = -log_of(P1, E1), sp = log_of(P2, E2);
      if (bad) atomicOr(a.status, ST_NOT_PD);
      if (a.mode == 0) {
        double v[5];
        combine5<double>(lr, sp, lsum, cmbv, v);
        if (bad)
          for (int q = 0; q < 5; q++) v[q] = __longlong_as_double(0x7ff8000000000000ll);
        store5<double>(a, gid, v);
      } else {
        b64[e] = bad ? __longlong_as_double(0x7ff8000000000000ll) : lr;
        b64[bstride + e] = sp;
        b64[2 * bstride + e] = lsum;
      }
    }
    __syncwarp(gmask);
  }
#undef AG
}

// Shared memory of the grouped kernel for (N, k) with G lanes per nplet and
// NT threads per block.
__host__ __device__ inline size_t f64g_smem(int N, int k, int NT, int G) {
  const SmemLayout L = smem_layout(N, k, row_stride(N), sizeof(double), 8, 0);
  const size_t per = (size_t)(k * (k + 1) / 2) * sizeof(double) + (size_t)k * sizeof(int);
  return L.total + per * (size_t)(NT / G) + 16;
}

}  // namespace thoi
