// Group objectives over D datasets (Results, "Leveraging Gaussian entropy
// estimators with batch processing": the nplet with the smallest average O
// across datasets; Methods, "Heuristics": the searches take several
// datasets; Methods, "fMRI analysis": the paired Cohen's d between two
// conditions).
//
// The per-dataset values of one measure come from each dataset's own nplet
// path (FP32 with the FP64 re-factor, or FP64) as one row of a D x ld matrix;
// these kernels fold the rows into the objective of every nplet:
//   mean    : g = (1/D) sum_d v_d
//   cohen_d : D = 2P, delta_i = v_i - v_{P+i}; g = mean(delta) / sd(delta),
//             sd with the P - 1 denominator (two passes over the P pairs)
// A nplet that is not positive definite in some dataset (NaN there), or whose
// differences all coincide (sd = 0), gets g = NaN: left out of reductions
// and counted as not positive definite.
#include <math.h>

#include "internal.cuh"
#include "nplet_common.cuh"

namespace thoi {

constexpr int GRP_NT = 256;

// Fold one dataset's status word and re-factor count into the group's, right
// after that dataset's pass (a context may appear more than once in a group,
// and its next pass resets both).
__global__ void k_group_fold(const int* status, const unsigned long long* flag_count,
                             unsigned long long flag_cap, int* gstatus,
                             unsigned long long* gnref) {
  // atomics: the datasets' passes (and their folds) run on several streams
  const int st = *status;
  if (st) atomicOr(gstatus, st);
  if (flag_count) {
    const unsigned long long f = *flag_count;
    atomicAdd(gnref, f < flag_cap ? f : flag_cap);
  }
}

__global__ void __launch_bounds__(GRP_NT)
    k_group_combine(const double* __restrict__ V, unsigned long long ld, unsigned long long n,
                    const unsigned long long* __restrict__ count, int D, int objective,
                    double* __restrict__ out, double* __restrict__ basis,
                    unsigned long long bstride) {
  if (count && *count < n) n = *count;  // a list whose length is known on the device
  const unsigned long long stride = (unsigned long long)gridDim.x * GRP_NT;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  for (unsigned long long i = (unsigned long long)blockIdx.x * GRP_NT + threadIdx.x; i < n;
       i += stride) {
    double g;
    if (objective == THOI_GROUP_MEAN) {
      double s = 0.0;
      for (int d = 0; d < D; d++) s += V[(size_t)d * ld + i];
      g = s / (double)D;
    } else {
      const int P = D / 2;
      double s = 0.0;
      for (int j = 0; j < P; j++) s += V[(size_t)j * ld + i] - V[(size_t)(P + j) * ld + i];
      const double m = s / (double)P;
      double q = 0.0;
      for (int j = 0; j < P; j++) {
        const double e = (V[(size_t)j * ld + i] - V[(size_t)(P + j) * ld + i]) - m;
        q = fma(e, e, q);
      }
      const double sd = sqrt(q / (double)(P - 1));
      g = sd > 0.0 ? m / sd : nan;  // NaN also when some value is NaN
    }
    if (out) out[i] = g;
    if (basis) {
      // basis triple whose combination (zero constants) gives H = TC = O = S = g
      basis[i] = -2.0 * g;
      basis[bstride + i] = 2.0 * g;
      basis[2 * bstride + i] = 4.0 * g;
    }
  }
}

// A candidate list shared by D datasets, replicated into D regions of stride
// cap_pad (the batched FP64 kernel reads each slot's list at its own offset),
// with the list length copied to every slot's counter.
__global__ void k_group_replicate(const unsigned long long* __restrict__ ids,
                                  const unsigned long long* __restrict__ count,
                                  unsigned long long cap, unsigned long long cap_pad,
                                  unsigned long long* __restrict__ ids_rep,
                                  unsigned long long* __restrict__ counts_rep) {
  const unsigned long long n = *count < cap ? *count : cap;
  const int d = blockIdx.y;
  if (blockIdx.x == 0 && threadIdx.x == 0) counts_rep[d] = n;
  for (unsigned long long e = (unsigned long long)blockIdx.x * GRP_NT + threadIdx.x; e < n;
       e += (unsigned long long)gridDim.x * GRP_NT)
    ids_rep[(size_t)d * cap_pad + e] = ids[e];
}

// One measure of every listed nplet of every dataset (grid.y = dataset) from
// the batched FP64 basis (dataset d's arrays at offset d * cap_pad, array
// stride lstride), into row d of the value matrix (row stride cap_pad).
__global__ void __launch_bounds__(GRP_NT)
    k_group_pick_batch(const double* __restrict__ b64, unsigned long long lstride,
                       unsigned long long cap_pad, const BatchSlot* __restrict__ slots,
                       const unsigned long long* __restrict__ count, int measure,
                       double* __restrict__ V) {
  const int d = blockIdx.y;
  const unsigned long long n = *count;
  const CombineV<double> cv(slots[d].cmb);
  const double* B = b64 + (size_t)d * cap_pad;
  double* row = V + (size_t)d * cap_pad;
  for (unsigned long long i = (unsigned long long)blockIdx.x * GRP_NT + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * GRP_NT) {
    const double lr = B[i];
    double v[5];
    combine5<double>(lr, B[lstride + i], B[2 * lstride + i], cv, v);
    row[i] = is_nan(lr) ? lr : pick5(v, measure);
  }
}

// Records of a group objective: every measure slot carries the objective's
// statistics (the reduction ran on a basis whose DTC slot is 0).
__global__ void k_group_fix(thoi_order_record* recs, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  thoi_order_record& r = recs[q];
  for (int m = 0; m < 5; m++) {
    r.min[m] = r.min[THOI_O];
    r.max[m] = r.max[THOI_O];
    r.mean[m] = r.mean[THOI_O];
    r.argmin[m] = r.argmin[THOI_O];
    r.argmax[m] = r.argmax[THOI_O];
  }
}

cudaError_t launch_group_fold(const int* status, const unsigned long long* flag_count,
                              unsigned long long flag_cap, int* gstatus, unsigned long long* gnref,
                              cudaStream_t s) {
  k_group_fold<<<1, 1, 0, s>>>(status, flag_count, flag_cap, gstatus, gnref);
  return cudaGetLastError();
}

cudaError_t launch_group_combine(const double* V, unsigned long long ld, unsigned long long n,
                                 const unsigned long long* count, int D, int objective,
                                 double* out, double* basis, unsigned long long bstride,
                                 int num_sms, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  long long grid = (long long)((n + GRP_NT - 1) / GRP_NT);
  if (grid > (long long)num_sms * 8) grid = (long long)num_sms * 8;
  k_group_combine<<<(unsigned)grid, GRP_NT, 0, s>>>(V, ld, n, count, D, objective, out, basis,
                                                    bstride);
  return cudaGetLastError();
}

cudaError_t launch_group_replicate(const unsigned long long* ids, const unsigned long long* count,
                                   unsigned long long cap, int D, unsigned long long cap_pad,
                                   unsigned long long* ids_rep, unsigned long long* counts_rep,
                                   cudaStream_t s) {
  if (D < 1 || D > 65535) return cudaErrorInvalidValue;
  long long bx = (long long)((cap + GRP_NT - 1) / GRP_NT);
  if (bx < 1) bx = 1;
  if (bx > 64) bx = 64;
  k_group_replicate<<<dim3((unsigned)bx, (unsigned)D), GRP_NT, 0, s>>>(ids, count, cap, cap_pad,
                                                                        ids_rep, counts_rep);
  return cudaGetLastError();
}

cudaError_t launch_group_pick_batch(const double* b64, unsigned long long lstride,
                                    unsigned long long cap_pad, int D, const BatchSlot* slots,
                                    const unsigned long long* count, unsigned long long cap,
                                    int measure, double* V, cudaStream_t s) {
  if (D < 1 || D > 65535) return cudaErrorInvalidValue;
  long long bx = (long long)((cap + GRP_NT - 1) / GRP_NT);
  if (bx < 1) bx = 1;
  if (bx > 64) bx = 64;
  k_group_pick_batch<<<dim3((unsigned)bx, (unsigned)D), GRP_NT, 0, s>>>(b64, lstride, cap_pad,
                                                                         slots, count, measure, V);
  return cudaGetLastError();
}

cudaError_t launch_group_fix(thoi_order_record* recs, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_group_fix<<<(n + 63) / 64, 64, 0, s>>>(recs, n);
  return cudaGetLastError();
}

}  // namespace thoi
