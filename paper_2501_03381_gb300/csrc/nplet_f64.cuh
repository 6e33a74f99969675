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
      bad |= !(d > 0.0);
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
