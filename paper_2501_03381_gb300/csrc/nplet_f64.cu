// FP64 nplet kernel: the THOI_F64 path and the re-factor of the nplets the
// FP32 path flagged.  One nplet per thread; each thread's k x k matrix lives
// in shared memory, interleaved across the block (entry e of thread t at
// mat[e * NT + t], so a warp's accesses to "its" entry are consecutive).
// FP64 arithmetic runs at a small fraction of the FP32 rate on this GPU, so
// shared-memory bandwidth is ample; what matters is latency, and shared
// memory keeps it far below that of per-thread local arrays.
//
// Same quantities as the FP32 kernels: R_S = Lh D Lh^T, log det R_S =
// sum log D_p, the unit-lower inverse V column by column, and
// p_j = (R_S^-1)_jj = 1/D_j + sum_{i>j} V_ij^2 / D_i.  A pivot D_p <= 0 marks
// the nplet not positive definite.
#include "nplet_common.cuh"

namespace thoi {

template <int NT, bool LIST, typename M>
__global__ void __launch_bounds__(NT) k_nplet_f64s(const NpletArgs a, double* __restrict__ b64,
                                                   unsigned long long bstride) {
  extern __shared__ __align__(16) unsigned char smem[];
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

template <int NT, bool LIST>
static cudaError_t launch_f64s_t(const NpletArgs& a, double* b64, unsigned long long bstride,
                                 size_t sm, int num_sms, cudaStream_t s, int* grid_out,
                                 int max_blocks) {
  void (*fn)(const NpletArgs, double*, unsigned long long);
  if (a.N > 32) fn = k_nplet_f64s<NT, LIST, unsigned long long>;
  else fn = k_nplet_f64s<NT, LIST, unsigned>;
  int occ = 0;
  cudaError_t e = occupancy_cached((const void*)fn, NT, sm, &occ);
  if (e != cudaSuccess) return e;
  long long grid = (long long)num_sms * occ;
  if (!LIST) {
    const unsigned long long n = a.rank_end - a.rank_begin;
    const long long need = (long long)((n + NT - 1) / NT);
    if (need < grid) grid = need > 0 ? need : 1;
  }
  if (grid > max_blocks) grid = max_blocks;
  fn<<<(unsigned)grid, NT, sm, s>>>(a, b64, bstride);
  if (grid_out) *grid_out = (int)grid;
  return cudaGetLastError();
}

// Threads per block so that the block's matrices fit in shared memory; 0 if
// even 32 matrices do not fit (the caller then uses the generic kernel).
int f64s_threads(int N, int k, size_t* smem_out) {
  const SmemLayout L = smem_layout(N, k, row_stride(N), sizeof(double), 8, 0);
  const size_t per = (size_t)(k * (k + 1) / 2) * sizeof(double);
  const size_t budget = 220 * 1024;
  for (int nt = 128; nt >= 32; nt >>= 1) {
    const size_t sm = L.total + per * nt;
    if (sm <= budget) {
      if (smem_out) *smem_out = sm;
      return nt;
    }
  }
  return 0;
}

// mode 0: five measures per nplet (SoA, per opt.out_f64); mode 2: basis
// values into b64 (3 arrays of bstride doubles, indexed by rank offset for
// the dense launch and by list position for the list launch).
cudaError_t launch_nplet_f64s(const NpletArgs& a, bool list, double* b64,
                              unsigned long long bstride, int num_sms, cudaStream_t s,
                              int* grid_out, int max_blocks) {
  size_t sm = 0;
  const int nt = f64s_threads(a.N, a.k, &sm);
  if (nt == 0) return cudaErrorInvalidValue;
  if (list) {
    if (nt == 128) return launch_f64s_t<128, true>(a, b64, bstride, sm, num_sms, s, grid_out, max_blocks);
    if (nt == 64) return launch_f64s_t<64, true>(a, b64, bstride, sm, num_sms, s, grid_out, max_blocks);
    return launch_f64s_t<32, true>(a, b64, bstride, sm, num_sms, s, grid_out, max_blocks);
  }
  if (nt == 128) return launch_f64s_t<128, false>(a, b64, bstride, sm, num_sms, s, grid_out, max_blocks);
  if (nt == 64) return launch_f64s_t<64, false>(a, b64, bstride, sm, num_sms, s, grid_out, max_blocks);
  return launch_f64s_t<32, false>(a, b64, bstride, sm, num_sms, s, grid_out, max_blocks);
}

}  // namespace thoi
