// Expansion step of the greedy search on the device (Methods, "Heuristics",
// "Greedy Algorithm"): every set selected at order k-1 grows by each variable
// it lacks, and the distinct candidates are listed by their lexicographic
// rank for the FP64 list evaluation.  With the selection, the evaluation and
// the expansion all on the stream, a whole search runs without a host round
// trip per order.
//
// Thread (i, v) takes parent i (entry i of the previous order's top list) and
// variable v.  Distinct candidates are kept by an open-addressing hash set of
// bit masks (0 = empty slot; a candidate has at least one bit) whose size is a
// power of two at least twice the number of candidates, so every probe
// sequence ends within the table.  The order of the list does not matter: the
// selection ranks by (value, rank).
#include "internal.cuh"

namespace thoi {

// 64-bit finaliser of MurmurHash3 (fmix64).
__device__ __forceinline__ unsigned long long gr_mix(unsigned long long x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}

__global__ void k_greedy_expand(const thoi_order_record* __restrict__ rec,
                                const TopEnt* __restrict__ tops, int kappa, int N, int kp,
                                const unsigned long long* __restrict__ binom,
                                unsigned long long* __restrict__ table, unsigned long long tsize,
                                unsigned long long* __restrict__ ids,
                                unsigned long long* __restrict__ count) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int i = (int)(t / N), v = (int)(t % N);
  if (i >= kappa) return;
  const int n = rec->top_count < kappa ? rec->top_count : kappa;
  if (i >= n) return;
  // the parent as a bit mask (bit c = variable c); unrank_mask gives bit N-1-c
  const unsigned long long rev = unrank_mask<unsigned long long>(tops[i].id, kp, N, binom);
  const unsigned long long parent = __brevll(rev) >> (64 - N);
  if (parent >> v & 1ull) return;
  const unsigned long long cand = parent | (1ull << v);
  unsigned long long h = gr_mix(cand) & (tsize - 1);
  for (unsigned long long probe = 0; probe < tsize; probe++) {
    const unsigned long long prev = atomicCAS(&table[h], 0ull, cand);
    if (prev == 0ull) {
      // first copy: list its lexicographic rank among the subsets of order kp + 1,
      // rank = C(N,k) - 1 - sum_i C(N-1-c_i, k-i) over the members c_0 < c_1 < ...
      const int k = kp + 1;
      unsigned long long rp = 0;
      int q = 0;
      for (unsigned long long m = cand; m; m &= m - 1, q++) {
        const int c = __ffsll((long long)m) - 1;
        rp += binom_at(binom, N - 1 - c, k - q);
      }
      ids[atomicAdd(count, 1ull)] = binom_at(binom, N, k) - 1ull - rp;
      return;
    }
    if (prev == cand) return;  // already listed
    h = (h + 1) & (tsize - 1);
  }
}

cudaError_t launch_greedy_expand(const thoi_order_record* rec, const TopEnt* tops, int kappa,
                                 int N, int kp, const unsigned long long* binom,
                                 unsigned long long* table, unsigned long long tsize,
                                 unsigned long long* ids, unsigned long long* count,
                                 cudaStream_t s) {
  if ((tsize & (tsize - 1)) != 0 || tsize < 2ull * (unsigned long long)kappa * N)
    return cudaErrorInvalidValue;
  const long long threads = (long long)kappa * N;
  const int nt = 256;
  k_greedy_expand<<<(unsigned)((threads + nt - 1) / nt), nt, 0, s>>>(rec, tops, kappa, N, kp, binom,
                                                                     table, tsize, ids, count);
  return cudaGetLastError();
}

}  // namespace thoi
