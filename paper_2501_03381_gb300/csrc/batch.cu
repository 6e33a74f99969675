// Multi-dataset batch: dispatch of the persistent batched FP32 nplet kernel
// by band of orders, and the batched FP64 re-factor and list-reduction
// kernels.  The bodies are those of the single-dataset kernels (f64s_body,
// f64g_body, reduce_core); here a block finds its dataset, order and range
// from descriptors in device memory instead of from launch arguments, so
// that one launch covers every dataset of the batch.
#include <type_traits>

#include "nplet_f64.cuh"
#include "reduce.cuh"

namespace thoi {

template <int KLO, int KHI>
cudaError_t bfused_launch(bool wide, const BatchFArgs& b, int maxN, int blocks_per_sm,
                          int num_sms, cudaStream_t s, int* grid_out);

cudaError_t launch_batch_fused(int band, bool wide, const BatchFArgs& b, int maxN,
                               int blocks_per_sm, int num_sms, cudaStream_t s, int* grid_out) {
  if (b.n_tiles <= 0) return cudaSuccess;
  switch (band) {
    case 0: return bfused_launch<1, 8>(wide, b, maxN, blocks_per_sm, num_sms, s, grid_out);
    case 1: return bfused_launch<9, 14>(wide, b, maxN, blocks_per_sm, num_sms, s, grid_out);
    case 2: return bfused_launch<15, 17>(wide, b, maxN, blocks_per_sm, num_sms, s, grid_out);
    case 3: return bfused_launch<18, 20>(wide, b, maxN, blocks_per_sm, num_sms, s, grid_out);
    default: return cudaErrorInvalidValue;
  }
}

static size_t reduce_smem(int top_m, size_t vsz, size_t isz) {
  return top_m > 0 ? (size_t)RTOP_CAP * 2 * (vsz + isz) : 0;
}

// ------------------------------------------------------------------ FP64 re-factor
// Block (x, y) re-factors list entries x, x + gridDim.x, ... (times NT) of
// slot slot0 + y in FP64 and writes their basis triples.
template <int NT, int G, typename M>
__global__ void __launch_bounds__(NT) k_refactor_batch(
    const BatchDataset* __restrict__ ds, const BatchSlot* __restrict__ slots, int slot0,
    const unsigned long long* __restrict__ binom, const unsigned long long* flag_ids,
    unsigned long long* flag_counts, double* __restrict__ b64, unsigned long long lstride,
    int* status) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int si = slot0 + blockIdx.y;
  const BatchSlot sl = slots[si];
  const BatchDataset D = ds[sl.d];
  NpletArgs a;
  a.N = D.N;
  a.k = sl.k;
  a.R32 = D.R32;
  a.R64 = D.R64;
  a.ls = D.ls;
  a.binom = binom;
  a.rank_begin = 0;
  a.rank_end = sl.n;
  a.id_base = sl.id_base;
  a.cmb = sl.cmb;
  a.tau_piv = D.tau_piv;
  a.tau_tr = D.tau_tr;
  a.mode = 2;
  a.out = nullptr;
  a.out_f64 = 1;
  a.out_sel = 0;
  a.out_n = 0;
  a.out_first = 0;
  a.part = nullptr;
  a.part_top = nullptr;
  a.top_m = 0;
  a.flag_ids = const_cast<unsigned long long*>(flag_ids) + sl.flag_off;
  a.flag_count = flag_counts + si;
  a.flag_cap = sl.flag_cap;
  a.status = status;
  a.cancel = nullptr;
  if constexpr (G == 1) f64s_body<NT, true, M>(a, b64 + sl.flag_off, lstride, smem);
  else f64g_body<NT, G, true, M>(a, b64 + sl.flag_off, lstride, smem);
}

template <int G, typename M>
static cudaError_t refactor_batch_t(const BatchDataset* ds, const BatchSlot* slots, int slot0,
                                    int n_slots, const unsigned long long* binom,
                                    const unsigned long long* flag_ids,
                                    unsigned long long* flag_counts, double* b64,
                                    unsigned long long lstride, int* status, int bx, size_t sm,
                                    cudaStream_t s) {
  constexpr int NT = 128;
  int occ = 0;
  cudaError_t e = occupancy_cached((const void*)k_refactor_batch<NT, G, M>, NT, sm, &occ);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)bx, (unsigned)n_slots);
  k_refactor_batch<NT, G, M><<<grid, NT, sm, s>>>(ds, slots, slot0, binom, flag_ids, flag_counts,
                                                  b64, lstride, status);
  return cudaGetLastError();
}

cudaError_t launch_refactor_batch(const BatchDataset* ds, const BatchSlot* slots, int slot0,
                                  int n_slots, int maxN, int k, bool wide,
                                  const unsigned long long* binom,
                                  const unsigned long long* flag_ids,
                                  unsigned long long* flag_counts, double* b64,
                                  unsigned long long lstride, int* status, int bx,
                                  cudaStream_t s) {
  if (n_slots <= 0) return cudaSuccess;
  if (bx < 1 || n_slots > 65535) return cudaErrorInvalidValue;
  // shared memory sized for the largest N (the layout grows with N)
  const F64Cfg c = f64_config(maxN, k);
#define RB(GG)                                                                                 \
  case GG:                                                                                     \
    return wide ? refactor_batch_t<GG, unsigned long long>(ds, slots, slot0, n_slots, binom,   \
                                                           flag_ids, flag_counts, b64, lstride, \
                                                           status, bx, c.smem, s)              \
                : refactor_batch_t<GG, unsigned>(ds, slots, slot0, n_slots, binom, flag_ids,   \
                                                 flag_counts, b64, lstride, status, bx, c.smem, \
                                                 s);
  switch (c.G) {
    RB(1) RB(2) RB(4) RB(8) RB(16) RB(32)
    default: return cudaErrorInvalidValue;
  }
#undef RB
}

// ------------------------------------------------------------------ list reduction
// Block (x, y) reduces list entries of slot slot0 + y into partial
// (slot0 + y) * gridDim.x + x.
__global__ void __launch_bounds__(RED_NT, 6) k_reduce_list_batch(
    const double* __restrict__ b64, unsigned long long lstride, const BatchSlot* __restrict__ slots,
    int slot0, const unsigned long long* __restrict__ flag_ids,
    const unsigned long long* flag_counts, int top_m, PartRec* __restrict__ part,
    TopEnt* __restrict__ part_top) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ RedScratch sc;
  __shared__ int s_tcnt[2];
  const int si = slot0 + blockIdx.y;
  const BatchSlot sl = slots[si];
  const double* B = b64 + sl.flag_off;
  const size_t pi = (size_t)si * gridDim.x + blockIdx.x;
  reduce_core<double, true>((unsigned long long)blockIdx.x * RED_NT + threadIdx.x,
                            (unsigned long long)gridDim.x * RED_NT, B, B + lstride, B + 2 * lstride,
                            0, flag_ids + sl.flag_off, flag_counts + si, sl.flag_cap, 0, sl.cmb,
                            top_m, 1, nullptr, part + pi, part_top + pi * 2 * top_m, smem, sc,
                            s_tcnt);
}

cudaError_t launch_reduce_list_batch(const double* b64, unsigned long long lstride,
                                     const BatchSlot* slots, int slot0, int n_slots,
                                     const unsigned long long* flag_ids,
                                     const unsigned long long* flag_counts, int top_m,
                                     PartRec* part, TopEnt* part_top, int bx, cudaStream_t s) {
  if (n_slots <= 0) return cudaSuccess;
  if (bx < 1 || n_slots > 65535) return cudaErrorInvalidValue;
  const size_t sm = reduce_smem(top_m, sizeof(double), sizeof(unsigned long long));
  int occ = 0;
  cudaError_t e = occupancy_cached((const void*)k_reduce_list_batch, RED_NT, sm, &occ);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)bx, (unsigned)n_slots);
  k_reduce_list_batch<<<grid, RED_NT, sm, s>>>(b64, lstride, slots, slot0, flag_ids, flag_counts,
                                               top_m, part, part_top);
  return cudaGetLastError();
}

}  // namespace thoi
