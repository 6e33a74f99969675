// Two-level prefix-shared FP32 nplet kernel for whole orders.  It extends
// the one-level kernel (nplet_pfx.cuh; the same bordered LDL^T steps) one
// level down: a thread factors a (k-2)-prefix G once, then for every middle
// index a > max(G) adds a as one stored bordered step, and for every last
// index b > a adds b as a final bordered step.  The nplets (G, a, b) of one
// (G, a) have consecutive ranks.
//
// Thread order: the (k-2)-prefixes are grouped by their largest index g;
// every prefix of a group runs the same nested loops (a over g+1 .. N-2, b
// over a+1 .. N-1), so the lanes of a warp stay together.
//
// PAIR: the final steps of two last indices b, b+1 run in one iteration.
// They share nothing but the factored (k-1)-prefix, so their dependency
// chains (forward solve, pivot, backward solve, products) interleave; with a
// thread's few warps per scheduler that is the latency the single step
// leaves exposed.
//
// DEPTH 3: a thread factors a (k-3)-prefix H once and, for every next index
// a1 > max(H), restores H's state and adds a1 as one stored bordered step,
// which yields the (k-2)-prefix of the loops above.  The rows of H's factor
// stay in place (a bordered step writes only its own row); H's inverse
// diagonal, which every step updates, is kept in shared memory.  A
// (k-2)-prefix then costs one step instead of a whole factorisation.
// DEPTH 4 adds one more such level: the thread factors a (k-4)-prefix I, and
// every next index a0 makes H = I + a0 by one stored step.
#pragma once
#include "nplet_common.cuh"

namespace thoi {

// Minimum resident blocks per SM: three (168 registers) up to order 14 at
// depth 2, measured 2-10% faster there despite a few spilled registers at 13
// and 14; above, and at depth 3 (one more saved state), the compiler's own
// allocation (up to 255 registers, two blocks).
template <int K, int DEPTH>
struct Pfx2Blocks {
  static constexpr int value = (K <= 14 && DEPTH == 2) ? 3 : 1;
};

template <int K, typename M, bool PAIR, int DEPTH>
__global__ void __launch_bounds__(RED_NT, Pfx2Blocks<K, DEPTH>::value)
    k_nplet_pfx2(const NpletArgs a, const int chunk) {
  static_assert(DEPTH == 2 || (DEPTH == 3 && K >= 5) || (DEPTH == 4 && K >= 6),
                "depth 2, depth 3 from order 5, depth 4 from order 6");
  constexpr int P = K - 1;   // variables before the last one
  constexpr int GP = K - 2;  // grand-prefix size
  constexpr int B0 = K - DEPTH;  // variables of the thread's own prefix (the grand prefix at depth 2)
  constexpr int BQ = B0 - 1;     // its indices below its largest index g
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
  // the threads' prefixes (largest index <= N-1-DEPTH)
  const unsigned long long T = binom_s(sb, bs, N - DEPTH, B0);
  const unsigned long long NK = binom_s(sb, bs, N, K);
  const unsigned long long nch = (T + chunk - 1) / chunk;
  const float tau_piv = a.tau_piv, tau_tr = a.tau_tr;
  const CombineV<float> cmbv(a.cmb);
  constexpr int MB = 8 * sizeof(M);

  float Lh[P][P];
  float dd[P], qd[P], qb[GP];
  // depth 3 and 4: the inverse diagonal of H, entry r of this thread at
  // qh[r * RED_NT]; depth 4: that of I after it (qi)
  float* const qh = reinterpret_cast<float*>(smem + (L.total + 15) / 16 * 16) + threadIdx.x;
  float* const qi = qh + (size_t)(K - 3) * RED_NT;
  constexpr int HB = K - 3;  // row of the step onto H (the index a1)
  int c[P];
  float P1 = 1.f, pmin = pinf<float>(), lsp = 0.f;
  int E1 = 0;
  bool badp = false;

  // Stored bordered step: variable ci joins the factored variables c[0..i-1]
  // as row i (Lh row i, dd[i], the inverse diagonal qd[0..i]).
  auto level = [&](const int i, const int ci) {
    const float* rowc = sR + ci * ldr;
    lsp += sls[ci];
    float x[P];
#pragma unroll
    for (int r = 0; r < i; r++) x[r] = rowc[c[r]];
#pragma unroll
    for (int r = 1; r < i; r++)
#pragma unroll
      for (int s = 0; s < r; s++) x[r] = fmaf(-Lh[r][s], x[s], x[r]);
    float Dn = rowc[ci];
#pragma unroll
    for (int r = 0; r < i; r++) {
      const float l = x[r] * dd[r];
      Dn = fmaf(-x[r], l, Dn);
      x[r] = l;
      Lh[i][r] = l;
    }
    pmin = fminf(pmin, Dn);
    P1 *= Dn;
    renorm(P1, E1, badp);
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
  };

  // Chunks of prefixes, 32 per warp at a time (consecutive chunks, so the
  // lanes share their prefixes' largest index): from the slot's work counter
  // when there is one (the work per prefix varies with its largest index,
  // and the heaviest groups come first), else a static split over the grid.
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
    int g = BQ;
    unsigned long long off = 0, gsz = binom_s(sb, bs, g, BQ);
    while (g0 >= off + gsz) {
      off += gsz;
      g++;
      gsz = binom_s(sb, bs, g, BQ);
    }
    unsigned long long j = g0 - off;
    M pm = unrank_s<M>(j, BQ, g, sb, bs);
    for (int jn = 0; jn < cnt; jn++) {
      {
        M t = pm;
#pragma unroll
        for (int q = 0; q < BQ; q++) {
          const int hb = hibit(t);
          t ^= (M)1 << hb;
          c[q] = g - 1 - hb;
        }
        c[BQ] = g;
      }
      // ---- the thread's prefix
      P1 = 1.f;
      E1 = 0;
      pmin = pinf<float>();
      lsp = 0.f;
      badp = false;
#pragma unroll
      for (int i = 0; i < B0; i++) level(i, c[i]);
      // ---- depth 4: every next index a0 as one stored step onto the thread's
      // prefix I, giving H (at depth 3, H is the thread's prefix)
      [[maybe_unused]] const float P1i = P1, pmini = pmin, lspi = lsp;
      [[maybe_unused]] const int E1i = E1;
      [[maybe_unused]] const bool badi = badp;
      if constexpr (DEPTH == 4) {
#pragma unroll
        for (int r = 0; r < B0; r++) qi[r * RED_NT] = qd[r];
      }
      const int a0_lo = DEPTH == 4 ? g + 1 : g;
      const int a0_hi = DEPTH == 4 ? N - 4 : g;
      for (int a0 = a0_lo; a0 <= a0_hi; a0++) {
      if constexpr (DEPTH == 4) {
        if (a0 > a0_lo) {
#pragma unroll
          for (int r = 0; r < B0; r++) qd[r] = qi[r * RED_NT];
          P1 = P1i;
          E1 = E1i;
          pmin = pmini;
          lsp = lspi;
          badp = badi;
        }
        c[B0] = a0;
        level(B0, a0);
      }
      // ---- depth 3 and 4: every next index a1 as one stored step onto H
      [[maybe_unused]] const float P1h = P1, pminh = pmin, lsph = lsp;
      [[maybe_unused]] const int E1h = E1;
      [[maybe_unused]] const bool badh = badp;
      if constexpr (DEPTH >= 3) {
#pragma unroll
        for (int r = 0; r < HB; r++) qh[r * RED_NT] = qd[r];
      }
      const int gh = DEPTH == 4 ? a0 : g;  // largest index of H (of the grand prefix at depth 2)
      const int a1_lo = DEPTH >= 3 ? gh + 1 : gh;
      const int a1_hi = DEPTH >= 3 ? N - 3 : gh;
      for (int a1 = a1_lo; a1 <= a1_hi; a1++) {
      if constexpr (DEPTH >= 3) {
        if (a1 > a1_lo) {
#pragma unroll
          for (int r = 0; r < HB; r++) qd[r] = qh[r * RED_NT];
          P1 = P1h;
          E1 = E1h;
          pmin = pminh;
          lsp = lsph;
          badp = badh;
        }
        c[HB] = a1;
        level(HB, a1);
      }
      // ---- grand prefix (largest index a1)
#pragma unroll
      for (int r = 0; r < GP; r++) qb[r] = qd[r];
      const float P1g = P1, pming = pmin, lspg = lsp;
      const int E1g = E1;
      const bool badg = badp;
      unsigned long long rbase = NK - 1ull;
#pragma unroll
      for (int i = 0; i < GP; i++) rbase -= binom_s(sb, bs, N - 1 - c[i], K - i);
      // ---- middle variables
      for (int am = a1 + 1; am < N - 1; am++) {
#pragma unroll
        for (int r = 0; r < GP; r++) qd[r] = qb[r];
        P1 = P1g;
        E1 = E1g;
        pmin = pming;
        lsp = lspg;
        badp = badg;
        c[GP] = am;
        level(GP, am);
        const unsigned long long r0 =
            rbase - binom_s(sb, bs, N - 1 - am, 2) - (unsigned long long)(N - 2 - am);
        // ---- last variables: one final bordered step each (two at a time
        // when PAIR: the two steps are independent, so their dependency
        // chains interleave)
        auto last = [&](const int cl, float& lr, float& sp, float& lsum, bool& bad) {
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
          bad = badp;
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
          lr = log_of(Pl, El);
          sp = log_of(P2, E2);
          lsum = lsp + sls[cl];
          bad |= !(fminf(pmin, Dn) >= tau_piv) | !(trace <= tau_tr);
        };
        auto emit = [&](const int cl, const float lr, const float sp, const float lsum,
                        const bool bad) {
          const unsigned long long gid = a.id_base + r0 + (unsigned long long)(cl - am - 1);
          if (fused) {
            fused_emit(a, acc, sthr, cmbv, gid, lr, sp, lsum, bad);
            return;
          }
          if (basis) {
            store_basis(a, gid, lr, sp, lsum, bad);
          } else {
            float v[5];
            combine5<float>(lr, sp, lsum, cmbv, v);
            store5<float>(a, gid, v);
          }
          flag_append(a, bad, gid);
        };
        if constexpr (PAIR) {
          for (int cl = am + 1; cl < N; cl += 2) {
            // an odd count repeats the last variable and drops the copy
            const int cl2 = cl + 1 < N ? cl + 1 : cl;
            float lr1, sp1, ls1, lr2, sp2, ls2;
            bool b1, b2;
            last(cl, lr1, sp1, ls1, b1);
            last(cl2, lr2, sp2, ls2, b2);
            emit(cl, lr1, sp1, ls1, b1);
            if (cl2 != cl) emit(cl2, lr2, sp2, ls2, b2);
          }
        } else {
          for (int cl = am + 1; cl < N; cl++) {
            float lr, sp, lsum;
            bool bad;
            last(cl, lr, sp, lsum, bad);
            emit(cl, lr, sp, lsum, bad);
          }
        }
      }
      }  // a1
      }  // a0
      if (jn + 1 < cnt) {
        if (j + 1 < gsz) {
          const M fullg = (g >= MB) ? ~(M)0 : (((M)1 << g) - 1);
          pm = lex_succ(pm, fullg);
          j++;
        } else {
          g++;
          gsz = binom_s(sb, bs, g, BQ);
          j = 0;
          pm = unrank_s<M>(0, BQ, g, sb, bs);
        }
      }
    }
  }
  if (fused) fused_block_end(a, acc);
}

// Shared memory of a launch: the tables, then (depth 3) the inverse diagonal
// of every thread's H.
template <int K, int DEPTH>
static size_t pfx2_smem(int N) {
  const SmemLayout L = smem_layout(N, K, row_stride(N), sizeof(float), sizeof(unsigned), 0);
  const size_t q = DEPTH == 3 ? (size_t)(K - 3) : (DEPTH == 4 ? (size_t)(2 * K - 7) : 0);
  return (L.total + 15) / 16 * 16 + q * RED_NT * sizeof(float);
}

template <int K, typename M, bool PAIR, int DEPTH>
static cudaError_t launch_pfx2_t(const NpletArgs& a, const Shape& sh, int num_sms,
                                 cudaStream_t s, int* grid_out, int max_blocks) {
  const size_t smem = pfx2_smem<K, DEPTH>(a.N);
  void (*fn)(const NpletArgs, const int) = k_nplet_pfx2<K, M, PAIR, DEPTH>;
  int occ = 0;
  cudaError_t e = occupancy_cached((const void*)fn, RED_NT, smem, &occ);
  if (e != cudaSuccess) return e;
  if (sh.blocks_per_sm > 0 && sh.blocks_per_sm < occ) occ = sh.blocks_per_sm;
  int chunk = sh.chunk > 0 ? sh.chunk : 1;
  if (chunk > 8) chunk = 8;
  // the threads' prefixes: C(N - DEPTH, K - DEPTH)
  unsigned __int128 t = 1;
  for (int i = 1; i <= K - DEPTH; i++) t = t * (unsigned)(a.N - K + i) / (unsigned)i;
  const unsigned long long T = (unsigned long long)t;
  long long grid = (long long)num_sms * occ;
  const long long need =
      (long long)((T + (unsigned long long)RED_NT * chunk - 1) / ((unsigned long long)RED_NT * chunk));
  if (need < grid) grid = need > 0 ? need : 1;
  if (grid > max_blocks) grid = max_blocks;
  fn<<<(unsigned)grid, RED_NT, smem, s>>>(a, chunk);
  if (grid_out) *grid_out = (int)grid;
  return cudaGetLastError();
}

// sh.prefix 2: two-level; 3: two-level with the last variables two at a
// time; 4: three-level (from order 5) and 5: four-level (from order 6), with
// the last variables two at a time
template <int K>
cudaError_t launch_pfx2_k(const NpletArgs& a, const Shape& sh, int num_sms, cudaStream_t s,
                          int* grid_out, int max_blocks) {
  const bool wide = a.N > 32;
  if constexpr (K >= 6) {
    if (sh.prefix == 5) {
      if (!wide) return launch_pfx2_t<K, unsigned, true, 4>(a, sh, num_sms, s, grid_out, max_blocks);
      return launch_pfx2_t<K, unsigned long long, true, 4>(a, sh, num_sms, s, grid_out, max_blocks);
    }
  }
  if constexpr (K >= 5) {
    if (sh.prefix >= 4) {
      if (!wide) return launch_pfx2_t<K, unsigned, true, 3>(a, sh, num_sms, s, grid_out, max_blocks);
      return launch_pfx2_t<K, unsigned long long, true, 3>(a, sh, num_sms, s, grid_out, max_blocks);
    }
  }
  if (sh.prefix >= 3) {
    if (!wide) return launch_pfx2_t<K, unsigned, true, 2>(a, sh, num_sms, s, grid_out, max_blocks);
    return launch_pfx2_t<K, unsigned long long, true, 2>(a, sh, num_sms, s, grid_out, max_blocks);
  }
  if (!wide) return launch_pfx2_t<K, unsigned, false, 2>(a, sh, num_sms, s, grid_out, max_blocks);
  return launch_pfx2_t<K, unsigned long long, false, 2>(a, sh, num_sms, s, grid_out, max_blocks);
}

}  // namespace thoi
