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
  const int st = *status;
  if (st) *gstatus |= st;
  if (flag_count) {
    const unsigned long long f = *flag_count;
    *gnref += f < flag_cap ? f : flag_cap;
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

// One measure of each listed nplet from its FP64 basis triple (NaN = not
// positive definite), into row `row` of the group matrix.
__global__ void __launch_bounds__(GRP_NT)
    k_group_pick(const double* __restrict__ b64, unsigned long long lstride,
                 const unsigned long long* __restrict__ count, Combine cmb, int measure,
                 double* __restrict__ row) {
  const unsigned long long n = *count;
  const CombineV<double> cv(cmb);
  for (unsigned long long i = (unsigned long long)blockIdx.x * GRP_NT + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * GRP_NT) {
    const double lr = b64[i];
    double v[5];
    combine5<double>(lr, b64[lstride + i], b64[2 * lstride + i], cv, v);
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

cudaError_t launch_group_pick(const double* b64, unsigned long long lstride,
                              const unsigned long long* count, unsigned long long cap,
                              Combine cmb, int measure, double* row, cudaStream_t s) {
  long long grid = (long long)((cap + GRP_NT - 1) / GRP_NT);
  if (grid < 1) grid = 1;
  if (grid > 1024) grid = 1024;
  k_group_pick<<<(unsigned)grid, GRP_NT, 0, s>>>(b64, lstride, count, cmb, measure, row);
  return cudaGetLastError();
}

cudaError_t launch_group_fix(thoi_order_record* recs, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_group_fix<<<(n + 63) / 64, 64, 0, s>>>(recs, n);
  return cudaGetLastError();
}

}  // namespace thoi
