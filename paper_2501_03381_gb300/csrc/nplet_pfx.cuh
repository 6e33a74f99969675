// Prefix-shared FP32 nplet kernel for whole orders.  The nplets of order k
// that share their first k-1 indices (a "prefix" whose largest index is m)
// differ only in the last index c, which runs over m+1 .. N-1; their ranks
// are consecutive.  A thread factors the prefix once and then adds each last
// variable as one bordered step, so a nplet costs O(k^2) instead of the
// O(k^3) of a full factorisation.
//
// Bordered LDL^T: with the prefix factorised as R_P = Lh D Lh^T, appending
// the variable c (column b_j = R[c][c_j], diagonal R[c][c]) gives
//   w = Lh^-1 b,  l = D^-1 w,  D_new = R[c][c] - w.l   (the new row of Lh is l)
// and, with V = Lh^-1, the new row of the inverse is v = -l^T V, i.e. the
// solution of Lh^T v = -l.  The inverse diagonal of the bordered matrix is
//   (R_S^-1)_jj = (R_P^-1)_jj + v_j^2 / D_new (j in P),  1 / D_new (new),
// and log det R_S = log det R_P + log D_new.  The prefix itself is built the
// same way, one variable at a time, keeping Lh, 1/D and (R_P^-1)_jj.
//
// Thread order: prefixes are grouped by their largest index m (all prefixes
// of a group have the same N-1-m last variables, so the lanes of a warp run
// loops of equal length); inside a group they are in lexicographic order of
// their first k-2 indices.  Results are written by global id, so the output
// is the same as the dense kernels' (the reduction reads it in rank order).
#pragma once
#include "nplet_common.cuh"

namespace thoi {

template <int K>
struct PfxBlocks {
  static constexpr int value = 1;
};

template <int K, typename M>
__global__ void __launch_bounds__(RED_NT, PfxBlocks<K>::value) k_nplet_pfx(const NpletArgs a,
                                                                          const int chunk) {
  constexpr int P = K - 1;  // prefix size
  constexpr int Q = K - 2;  // prefix indices below its largest index m
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = a.N, ldr = row_stride(N);
  const SmemLayout L = smem_layout(N, K, ldr, sizeof(float), sizeof(unsigned), 0);
  load_tables<float>(a, smem, L, a.R32);
  const unsigned long long* sb = reinterpret_cast<const unsigned long long*>(smem + L.binom);
  const float* sR = reinterpret_cast<const float*>(smem + L.R);
  const float* sls = reinterpret_cast<const float*>(smem + L.ls);
  constexpr int bs = K + 1;
  const bool basis = a.mode == 2;
  const bool fused = a.mode == 3;
  const float* sthr = reinterpret_cast<const float*>(smem + L.thr);
  FusedAcc acc;
  acc.init();
  const unsigned long long T = binom_s(sb, bs, N - 1, P);  // prefixes (largest index <= N-2)
  const unsigned long long NK = binom_s(sb, bs, N, K);
  const unsigned long long nch = (T + chunk - 1) / chunk;
  const float tau_piv = a.tau_piv, tau_tr = a.tau_tr;
  const CombineV<float> cmbv(a.cmb);
  constexpr int MB = 8 * sizeof(M);

  // Chunks of prefixes, 32 per warp at a time (consecutive chunks, so the
  // lanes share their prefixes' largest index): from the slot's work counter
  // when there is one, else a static split over the grid.
  const int lane = threadIdx.x & 31;
  for (unsigned it = 0;; it++) {
    unsigned long long wb = 0;
    int stop = 0;
    if (lane == 0) {
      wb = a.work_counter ? atomicAdd(a.work_counter, 32ull)
                          : (((unsigned long long)it * gridDim.x + blockIdx.x) * (RED_NT / 32) +
                             (threadIdx.x >> 5)) * 32ull;
      stop = (it & 63) == 63 && a.cancel && *(volatile const int*)a.cancel;
    }
    wb = __shfl_sync(0xffffffffu, wb, 0);
    stop = __shfl_sync(0xffffffffu, stop, 0);
    if (stop) {
      if (lane == 0) atomicOr(a.status, ST_CANCELLED);
      break;
    }
    if (wb >= nch) break;
    const unsigned long long ch = wb + (unsigned long long)lane;
    if (ch >= nch) continue;
    const unsigned long long g0 = ch * chunk;
    const int cnt = T - g0 < (unsigned long long)chunk ? (int)(T - g0) : chunk;
    // group (largest prefix index m) of prefix g0 and its rank j inside the group
    int m = Q;
    unsigned long long off = 0, gsz = binom_s(sb, bs, m, Q);
    while (g0 >= off + gsz) {
      off += gsz;
      m++;
      gsz = binom_s(sb, bs, m, Q);
    }
    unsigned long long j = g0 - off;
    // first Q indices: a Q-subset of {0..m-1}, reversed mask in that universe
    M pm = unrank_s<M>(j, Q, m, sb, bs);
    for (int jn = 0; jn < cnt; jn++) {
      int c[P];
      {
        M t = pm;
#pragma unroll
        for (int q = 0; q < Q; q++) {
          const int hb = hibit(t);
          t ^= (M)1 << hb;
          c[q] = m - 1 - hb;
        }
        c[Q] = m;
      }
      // ---- prefix: Lh (strictly lower), dd = 1/D, qd = (R_P^-1)_jj
      float Lh[P][P];
      float dd[P], qd[P];
      float P1 = 1.f, pmin = pinf<float>(), lsp = 0.f;
      int E1 = 0;
      bool badp = false;
#pragma unroll
      for (int i = 0; i < P; i++) {
        const float* rowc = sR + c[i] * ldr;
        lsp += sls[c[i]];
        float x[P];
#pragma unroll
        for (int r = 0; r < i; r++) x[r] = rowc[c[r]];
#pragma unroll
        for (int r = 1; r < i; r++)
#pragma unroll
          for (int s = 0; s < r; s++) x[r] = fmaf(-Lh[r][s], x[s], x[r]);
        float Dn = rowc[c[i]];
#pragma unroll
        for (int r = 0; r < i; r++) {
          const float l = x[r] * dd[r];
          Dn = fmaf(-x[r], l, Dn);
          x[r] = l;
          Lh[i][r] = l;
        }
        pmin = fminf(pmin, Dn);
        P1 *= Dn;
        if ((i & 3) == 3 || i == P - 1) renorm(P1, E1, badp);
        const float dn = rcp_approx(Dn);
        dd[i] = dn;
#pragma unroll
        for (int r = i - 1; r >= 0; r--) {
          float s = -x[r];
          // x[r + 1], the latest finished, enters last: each x[r] then waits one FMA for it
#pragma unroll
          for (int t = i - 1; t > r; t--) s = fmaf(-Lh[t][r], x[t], s);
          x[r] = s;
        }
#pragma unroll
        for (int r = 0; r < i; r++) qd[r] = fmaf(x[r] * dn, x[r], qd[r]);
        qd[i] = dn;
      }
      // rank of (prefix, m + 1): r' = sum_i C(N-1-c_i, k-i), rank = C(N,k)-1-r'
      unsigned long long rp = (unsigned long long)(N - 2 - m);
#pragma unroll
      for (int i = 0; i < P; i++) rp += binom_s(sb, bs, N - 1 - c[i], K - i);
      const unsigned long long r0 = NK - 1ull - rp;
      // ---- one bordered step per last variable
      for (int cl = m + 1; cl < N; cl++) {
        const float* rowc = sR + cl * ldr;
        float x[P];
#pragma unroll
        for (int r = 0; r < P; r++) x[r] = rowc[c[r]];
#pragma unroll
        for (int r = 1; r < P; r++)
#pragma unroll
          for (int s = 0; s < r; s++) x[r] = fmaf(-Lh[r][s], x[s], x[r]);
        float Dn = rowc[cl];
#pragma unroll
        for (int r = 0; r < P; r++) {
          const float l = x[r] * dd[r];
          Dn = fmaf(-x[r], l, Dn);
          x[r] = l;
        }
        const float dn = rcp_approx(Dn);
#pragma unroll
        for (int r = P - 1; r >= 0; r--) {
          float s = -x[r];
          // x[r + 1], the latest finished, enters last: each x[r] then waits one FMA for it
#pragma unroll
          for (int t = P - 1; t > r; t--) s = fmaf(-Lh[t][r], x[t], s);
          x[r] = s;
        }
        bool bad = badp;
        float Pl = P1 * Dn;
        int El = E1;
        renorm(Pl, El, bad);
        float P2 = dn, trace = dn;
        int E2 = 0;
        // in the order the backward solve finishes the x[r] (descending), so the
        // product and the trace overlap with it
#pragma unroll
        for (int r = P - 1; r >= 0; r--) {
          const float pr = fmaf(x[r] * dn, x[r], qd[r]);
          trace += pr;
          P2 *= pr;
          if (((P - 1 - r) & 3) == 3 || r == 0) renorm(P2, E2, bad);
        }
        const float lr = log_of(Pl, El), sp = log_of(P2, E2);
        const float lsum = lsp + sls[cl];
        bad |= !(fminf(pmin, Dn) >= tau_piv) | !(trace <= tau_tr);
        const unsigned long long gid = a.id_base + r0 + (unsigned long long)(cl - m - 1);
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
      // next prefix: lexicographic successor inside the group, or the first
      // prefix of the next group
      if (jn + 1 < cnt) {
        if (j + 1 < gsz) {
          const M fullm = (m >= MB) ? ~(M)0 : (((M)1 << m) - 1);
          pm = lex_succ(pm, fullm);
          j++;
        } else {
          m++;
          gsz = binom_s(sb, bs, m, Q);
          j = 0;
          pm = unrank_s<M>(0, Q, m, sb, bs);
        }
      }
    }
  }
  if (fused) fused_block_end(a, acc);
}

template <int K, typename M>
static cudaError_t launch_pfx_t(const NpletArgs& a, const Shape& sh, int num_sms, cudaStream_t s,
                                int* grid_out, int max_blocks) {
  const SmemLayout L = smem_layout(a.N, K, row_stride(a.N), sizeof(float), sizeof(unsigned), 0);
  void (*fn)(const NpletArgs, const int) = k_nplet_pfx<K, M>;
  int occ = 0;
  cudaError_t e = occupancy_cached((const void*)fn, RED_NT, L.total, &occ);
  if (e != cudaSuccess) return e;
  if (sh.blocks_per_sm > 0 && sh.blocks_per_sm < occ) occ = sh.blocks_per_sm;
  int chunk = sh.chunk > 0 ? sh.chunk : 2;
  if (chunk > 8) chunk = 8;
  // prefixes of the order: C(N-1, K-1)
  unsigned __int128 t = 1;
  for (int i = 1; i <= K - 1; i++) t = t * (unsigned)(a.N - K + i) / (unsigned)i;
  const unsigned long long T = (unsigned long long)t;
  long long grid = (long long)num_sms * occ;
  const long long need =
      (long long)((T + (unsigned long long)RED_NT * chunk - 1) / ((unsigned long long)RED_NT * chunk));
  if (need < grid) grid = need > 0 ? need : 1;
  if (grid > max_blocks) grid = max_blocks;
  fn<<<(unsigned)grid, RED_NT, L.total, s>>>(a, chunk);
  if (grid_out) *grid_out = (int)grid;
  return cudaGetLastError();
}

template <int K>
cudaError_t launch_pfx_k(const NpletArgs& a, const Shape& sh, int num_sms, cudaStream_t s,
                         int* grid_out, int max_blocks) {
  if (a.N <= 32) return launch_pfx_t<K, unsigned>(a, sh, num_sms, s, grid_out, max_blocks);
  return launch_pfx_t<K, unsigned long long>(a, sh, num_sms, s, grid_out, max_blocks);
}

}  // namespace thoi
