// Simulated annealing over nplets (Methods, "Heuristics", "Simulated
// Annealing Algorithm").  Every chain runs the whole schedule on the device
// (a thread, or a warp, per chain; see below): propose a neighbour of its
// current set, evaluate its energy in FP64, accept by the Metropolis rule,
// cool.  Chains are independent, so the kernels need no communication
// between chains and no host round trip.
//
// Random numbers: draw (chain, iteration, slot) is output number
// c = (chain * (iters + 1) + iteration) * 64 + slot of the SplitMix64
// generator seeded with `seed`, i.e. the SplitMix64 finaliser applied to
// seed + (c + 1) * 0x9E3779B97F4A7C15 (mod 2^64).  Integers in [0, n) are
// (z * n) >> 64; uniforms in [0, 1) are (z >> 11) * 2^-53.
//
// Moves (the paper does not fix them): within one order (k_lo == k_hi) a
// swap of a member (draw 1) with a non-member (draw 2); across orders, draw 0
// picks a variable that is added (if absent and the set is below k_hi) or
// removed (if present and the set is above k_lo), else the move is a swap.
// Acceptance: always if the energy rises, else with probability
// exp(dE / Temp) (the paper prints exp(-dE / Temp), which is at least 1 for
// dE <= 0; the sign is read as the usual Metropolis rule).  Temp = T0 at step
// 1, multiplied by alpha after every step.  Termination (the paper's two
// criteria): after `iters` steps, or, with patience > 0, after the first step
// t with no rise of the best energy since step t - patience.  Energy = the
// measure (maximise) or its negative (minimise); sets that are not positive
// definite are rejected.  Over D > 1 datasets the value is a group objective
// (Methods, "Heuristics": the searches take several datasets): the mean of
// the measure, or the paired Cohen's d (datasets i and P + i paired; mean
// and spread of the differences in two passes).  A group chain is one warp:
// every lane runs the same schedule and draws, and the lanes share the
// datasets of each evaluation (warp sums are butterflies, so every lane holds
// the same bits and the warp never diverges on an acceptance).  One dataset
// with fewer chains than lanes can fill (below SA_WARP_CHAINS) also runs a
// warp per chain: the 32 lanes share each factorisation, a row per lane.
#include <math.h>

#include "internal.cuh"
#include "nplet_common.cuh"
#include "nplet_f64.cuh"

namespace thoi {

constexpr int SA_KMAX = 32;
constexpr int SA_NT = 64;

__device__ __forceinline__ unsigned long long sm64(unsigned long long seed, unsigned long long c) {
  unsigned long long z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ int draw_int(unsigned long long z, int n) {
  return (int)__umul64hi(z, (unsigned long long)n);
}
__device__ __forceinline__ double draw_unit(unsigned long long z) {
  return (double)(z >> 11) * 0x1.0p-53;
}

// i-th member (ascending) of mask m, i < popcount
__device__ __forceinline__ int nth_member(unsigned long long m, int i) {
  for (int q = 0; q < i; q++) m &= m - 1;
  return __ffsll((long long)m) - 1;
}

// FP64 measure of the set `mask` (|mask| = k <= SA_KMAX): LDL^T of R_S, unit
// lower inverse, inverse diagonal; NaN when R_S is not positive definite.
__device__ double sa_measure(unsigned long long mask, const double* sR, int ldr, const double* sls,
                             const Combine* cmb, int measure) {
  int c[SA_KMAX];
  int k = 0;
  for (unsigned long long m = mask; m; m &= m - 1) c[k++] = __ffsll((long long)m) - 1;
  double A[SA_KMAX * (SA_KMAX + 1) / 2];
#define SA(i, j) A[((i) * ((i) + 1)) / 2 + (j)]
  double lsum = 0.0;
  for (int i = 0; i < k; i++) {
    lsum += sls[c[i]];
    for (int j = 0; j <= i; j++) SA(i, j) = sR[c[i] * ldr + c[j]];
  }
  double P1 = 1.0, P2 = 1.0;
  int E1 = 0, E2 = 0;
  bool bad = false;
  for (int p = 0; p < k; p++) {
    const double d = SA(p, p);
    bad |= !pivot_ok(d);
    P1 *= d;
    renorm(P1, E1, bad);
    const double rd = 1.0 / d;
    SA(p, p) = rd;
    for (int i = k - 1; i > p; i--) {
      const double u = SA(i, p) * rd;
      for (int j = p + 1; j <= i; j++) SA(i, j) = fma(-u, SA(j, p), SA(i, j));
      SA(i, p) = u;
    }
  }
  for (int j = 0; j < k; j++) {
    double pj = SA(j, j);
    for (int i = j + 1; i < k; i++) {
      double s = SA(i, j);
      for (int q = j + 1; q < i; q++) s = fma(-SA(i, q), SA(q, j), s);
      SA(i, j) = s;
      pj = fma(s * SA(i, i), s, pj);
    }
    P2 *= pj;
    renorm(P2, E2, bad);
  }
#undef SA
  if (bad) return __longlong_as_double(0x7ff8000000000000ll);
  const double lr = log_of(P1, E1), sp = log_of(P2, E2);
  const CombineV<double> cv(cmb[k]);
  double v[5];
  combine5<double>(lr, sp, lsum, cv, v);
  return pick5(v, measure);
}

// The whole schedule of one chain (start, moves, Metropolis acceptance,
// cooling); value(mask) is the measure or group objective of a set.  Every
// caller thread of a chain runs it identically; `write` selects the one that
// stores the results.
template <typename F>
__device__ __forceinline__ void sa_chain(const int chain, const int N, const int klo,
                                         const int khi, const int iters, const double T0,
                                         const double alpha, const int patience,
                                         const int maximize,
                                         const unsigned long long seed, F&& value,
                                         const bool write, unsigned long long* final_mask,
                                         double* final_val, unsigned long long* best_mask,
                                         double* best_val, unsigned long long* accepted) {
  const unsigned long long base = (unsigned long long)chain * (unsigned long long)(iters + 1);
  auto draw = [&](int it, int slot) { return sm64(seed, (base + it) * 64ull + slot); };
  const double sgn = maximize ? 1.0 : -1.0;
  // initial set: size klo + draw, members by a partial Fisher-Yates shuffle
  unsigned long long mask = 0;
  {
    const int size = klo + draw_int(draw(0, 0), khi - klo + 1);
    int perm[THOI_MAX_N];
    for (int v = 0; v < N; v++) perm[v] = v;
    for (int j = 0; j < size; j++) {
      const int r = j + draw_int(draw(0, 1 + j), N - j);
      const int t = perm[j];
      perm[j] = perm[r];
      perm[r] = t;
      mask |= 1ull << perm[j];
    }
  }
  double E = sgn * value(mask);
  double bestE = E;
  unsigned long long bmask = mask;
  double T = T0;
  int t_best = 0;  // last step that raised the best energy
  unsigned long long acc = 0;
  const unsigned long long full = N >= 64 ? ~0ull : ((1ull << N) - 1ull);
  for (int it = 1; it <= iters; it++) {
    const int size = __popcll(mask);
    unsigned long long prop = mask;
    bool swap = klo == khi;
    if (!swap) {
      const int v = draw_int(draw(it, 0), N);
      const bool in = mask >> v & 1ull;
      if (!in && size < khi) prop = mask | (1ull << v);
      else if (in && size > klo) prop = mask & ~(1ull << v);
      else swap = true;
    }
    if (swap && size < N) {
      const int v = nth_member(mask, draw_int(draw(it, 1), size));
      const int w = nth_member(~mask & full, draw_int(draw(it, 2), N - size));
      prop = (mask & ~(1ull << v)) | (1ull << w);
    }
    const double En = sgn * value(prop);
    if (En == En) {
      const double dE = En - E;
      bool ok = dE > 0.0;
      if (!ok) {
        const double p = dE == 0.0 ? 1.0 : exp(dE / T);
        ok = draw_unit(draw(it, 3)) < p;
      }
      if (ok) {
        mask = prop;
        E = En;
        acc++;
        if (E > bestE) {
          bestE = E;
          bmask = mask;
          t_best = it;
        }
      }
    }
    T *= alpha;
    // early stop: no improvement of the best energy for `patience` steps
    // (every thread of a chain holds the same t_best, so a warp stops together)
    if (patience > 0 && it - t_best >= patience) break;
  }
  if (write) {
    final_mask[chain] = mask;
    final_val[chain] = sgn * E;
    best_mask[chain] = bmask;
    best_val[chain] = sgn * bestE;
    accepted[chain] = acc;
  }
}

// One dataset: a thread per chain, the tables in shared memory.
__global__ void __launch_bounds__(SA_NT) k_anneal(const double* __restrict__ R64,
                                                  const double* __restrict__ ls, int N, int klo,
                                                  int khi, const Combine* __restrict__ cmb_tab,
                                                  int n_chains, int iters, double T0, double alpha,
                                                  int patience, int measure, int maximize,
                                                  unsigned long long seed,
                                                  unsigned long long* __restrict__ final_mask,
                                                  double* __restrict__ final_val,
                                                  unsigned long long* __restrict__ best_mask,
                                                  double* __restrict__ best_val,
                                                  unsigned long long* __restrict__ accepted) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int ldr = row_stride(N);
  double* sR = reinterpret_cast<double*>(smem);
  double* sls = sR + (size_t)N * ldr;
  Combine* scmb = reinterpret_cast<Combine*>(sls + N);
  for (int q = threadIdx.x; q < N * N; q += blockDim.x) sR[(q / N) * ldr + (q % N)] = R64[q];
  for (int q = threadIdx.x; q < N; q += blockDim.x) sls[q] = ls[q];
  for (int q = threadIdx.x; q <= khi; q += blockDim.x) scmb[q] = cmb_tab[q];
  __syncthreads();
  const int chain = blockIdx.x * blockDim.x + threadIdx.x;
  if (chain >= n_chains) return;
  sa_chain(chain, N, klo, khi, iters, T0, alpha, patience, maximize, seed,
           [&](unsigned long long m) { return sa_measure(m, sR, ldr, sls, scmb, measure); }, true,
           final_mask, final_val, best_mask, best_val, accepted);
}

constexpr int SA_GNT = 128;            // warp-per-chain kernels: four chains per block
constexpr int SA_WARP_CHAINS = 16384;  // one dataset: a warp per chain below this many chains

// One dataset, a warp per chain: the chain's k x k triangle and member list
// in shared memory, row i on lane i (k <= 32), factorised by the 32 lanes
// together (f64g_factor); every lane ends with the same value.
__global__ void __launch_bounds__(SA_GNT)
    k_anneal_warp(const double* __restrict__ R64, const double* __restrict__ ls, int N, int klo,
                  int khi, const Combine* __restrict__ cmb_tab, int n_chains, int iters, double T0,
                  double alpha, int patience, int measure, int maximize, unsigned long long seed,
                  unsigned long long* __restrict__ final_mask, double* __restrict__ final_val,
                  unsigned long long* __restrict__ best_mask, double* __restrict__ best_val,
                  unsigned long long* __restrict__ accepted) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int ldr = row_stride(N);
  double* sR = reinterpret_cast<double*>(smem);
  double* sls = sR + (size_t)N * ldr;
  Combine* scmb = reinterpret_cast<Combine*>(sls + N);
  const int tri = khi * (khi + 1) / 2;
  double* A = reinterpret_cast<double*>(scmb + khi + 1) + (size_t)(threadIdx.x >> 5) * tri;
  int* C = reinterpret_cast<int*>(reinterpret_cast<double*>(scmb + khi + 1) +
                                  (size_t)(SA_GNT / 32) * tri) +
           (threadIdx.x >> 5) * khi;
  for (int q = threadIdx.x; q < N * N; q += blockDim.x) sR[(q / N) * ldr + (q % N)] = R64[q];
  for (int q = threadIdx.x; q < N; q += blockDim.x) sls[q] = ls[q];
  for (int q = threadIdx.x; q <= khi; q += blockDim.x) scmb[q] = cmb_tab[q];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int chain = (int)(((unsigned)blockIdx.x * SA_GNT + threadIdx.x) >> 5);
  if (chain >= n_chains) return;  // whole warps leave together
#define AG(i, j) A[((((i) * ((i) + 1)) >> 1) + (j))]
  auto value = [&](unsigned long long mask) -> double {
    const int k = __popcll(mask);
    if (lane < k) C[lane] = nth_member(mask, lane);
    __syncwarp();
    double lsum = 0.0;
    if (lane < k) {
      const int ci = C[lane];
      const double* row = sR + ci * ldr;
      lsum = sls[ci];
      for (int j = 0; j <= lane; j++) AG(lane, j) = row[C[j]];
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    __syncwarp();
    double P1 = 1.0, P2 = 1.0;
    int E1 = 0, E2 = 0;
    bool bad = false;
    f64g_factor<32>(A, k, lane, 0xffffffffu, P1, E1, P2, E2, bad);
    bad = __any_sync(0xffffffffu, bad);
    const double lr = __shfl_sync(0xffffffffu, -log_of(P1, E1), 0);
    __syncwarp();  // the triangle is rewritten by the next evaluation
    if (bad) return __longlong_as_double(0x7ff8000000000000ll);
    const double sp = log_of(P2, E2);
    const CombineV<double> cv(scmb[k]);
    double v[5];
    combine5<double>(lr, sp, lsum, cv, v);
    return pick5(v, measure);
  };
#undef AG
  sa_chain(chain, N, klo, khi, iters, T0, alpha, patience, maximize, seed, value, lane == 0, final_mask,
           final_val, best_mask, best_val, accepted);
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// D > 1 datasets: a warp per chain.  Lane L evaluates datasets L, L + 32, ...
// For Cohen's d the datasets are taken in pair order h = 2j + side (side 0:
// dataset j, condition A; side 1: dataset P + j), so the two sides of a pair
// sit on neighbouring lanes and one shuffle forms the difference.
__global__ void __launch_bounds__(SA_GNT)
    k_anneal_group(const double* const* __restrict__ Rs, const double* const* __restrict__ lss,
                   int D, int objective, int N, int klo, int khi,
                   const Combine* __restrict__ cmb_tab, int n_chains, int iters, double T0,
                   double alpha, int patience, int measure, int maximize, unsigned long long seed,
                   unsigned long long* __restrict__ final_mask, double* __restrict__ final_val,
                   unsigned long long* __restrict__ best_mask, double* __restrict__ best_val,
                   unsigned long long* __restrict__ accepted) {
  const int lane = threadIdx.x & 31;
  const int chain = (int)(((unsigned)blockIdx.x * SA_GNT + threadIdx.x) >> 5);
  if (chain >= n_chains) return;  // whole warps leave together
  const int ncmb = khi + 1, rounds = (D + 31) / 32, P = D / 2;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  auto one = [&](unsigned long long m, int d) {
    return sa_measure(m, Rs[d], N, lss[d], cmb_tab + (size_t)d * ncmb, measure);
  };
  auto value = [&](unsigned long long m) -> double {
    if (objective == THOI_GROUP_MEAN) {
      double s = 0.0;
      for (int q = 0; q < rounds; q++) {
        const int d = lane + 32 * q;
        s += d < D ? one(m, d) : 0.0;
      }
      return warp_sum(s) / (double)D;
    }
    double dl[THOI_MAX_GROUP / 32];  // this lane's differences (even lanes)
    double s = 0.0;
    for (int q = 0; q < rounds; q++) {
      const int h = lane + 32 * q;
      const double v = h < D ? one(m, (h & 1) ? P + (h >> 1) : (h >> 1)) : 0.0;
      const double w = __shfl_xor_sync(0xffffffffu, v, 1);
      dl[q] = (h < D && !(h & 1)) ? v - w : 0.0;
      s += dl[q];
    }
    const double mean = warp_sum(s) / (double)P;
    double ss = 0.0;
    for (int q = 0; q < rounds; q++) {
      const int h = lane + 32 * q;
      const double e = (h < D && !(h & 1)) ? dl[q] - mean : 0.0;
      ss = fma(e, e, ss);
    }
    const double sd = sqrt(warp_sum(ss) / (double)(P - 1));
    return sd > 0.0 ? mean / sd : nan;
  };
  sa_chain(chain, N, klo, khi, iters, T0, alpha, patience, maximize, seed, value, lane == 0, final_mask,
           final_val, best_mask, best_val, accepted);
}

cudaError_t launch_anneal(const double* const* Rs, const double* const* lss, int D,
                          int objective, int N, int klo, int khi, const Combine* cmb_tab,
                          const double* R0, const double* ls0, int n_chains, int iters, double T0,
                          double alpha, int patience, int measure, int maximize,
                          unsigned long long seed,
                          unsigned long long* final_mask, double* final_val,
                          unsigned long long* best_mask, double* best_val,
                          unsigned long long* accepted, cudaStream_t s) {
  if (khi > SA_KMAX || klo < 1 || khi < klo || khi > N || n_chains < 1 || iters < 0 || D < 1 ||
      D > THOI_MAX_GROUP || patience < 0)
    return cudaErrorInvalidValue;
  if (D == 1 && n_chains < SA_WARP_CHAINS) {
    const size_t sm = ((size_t)N * row_stride(N) + N) * sizeof(double) +
                      (size_t)(khi + 1) * sizeof(Combine) +
                      (size_t)(SA_GNT / 32) * ((size_t)khi * (khi + 1) / 2 * sizeof(double) +
                                               (size_t)khi * sizeof(int));
    const long long threads = (long long)n_chains * 32;
    const int grid = (int)((threads + SA_GNT - 1) / SA_GNT);
    if (sm > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(
          k_anneal_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    k_anneal_warp<<<grid, SA_GNT, sm, s>>>(R0, ls0, N, klo, khi, cmb_tab, n_chains, iters, T0,
                                           alpha, patience, measure, maximize, seed, final_mask, final_val,
                                           best_mask, best_val, accepted);
    return cudaGetLastError();
  }
  if (D == 1) {
    const size_t sm = ((size_t)N * row_stride(N) + N) * sizeof(double) +
                      (size_t)(khi + 1) * sizeof(Combine);
    const int grid = (n_chains + SA_NT - 1) / SA_NT;
    k_anneal<<<grid, SA_NT, sm, s>>>(R0, ls0, N, klo, khi, cmb_tab, n_chains, iters, T0, alpha,
                                     patience, measure, maximize, seed, final_mask, final_val, best_mask,
                                     best_val, accepted);
    return cudaGetLastError();
  }
  const long long threads = (long long)n_chains * 32;
  const int grid = (int)((threads + SA_GNT - 1) / SA_GNT);
  k_anneal_group<<<grid, SA_GNT, 0, s>>>(Rs, lss, D, objective, N, klo, khi, cmb_tab, n_chains,
                                         iters, T0, alpha, patience, measure, maximize, seed,
                                         final_mask,
                                         final_val, best_mask, best_val, accepted);
  return cudaGetLastError();
}

}  // namespace thoi
