// Entry point that allocates no device memory: the per-order reduction of
// one order k in the FP64 path, with every piece of scratch it needs
// (correlation matrix, log-variances, binomial table, per-block partial
// records and top lists, status word) carved from one fixed, file-scope
// device array.
//
// Who needs this: callers that cannot call cudaMalloc or cudaFree.  For
// example, an application whose device memory is entirely owned by another
// allocator (a framework's caching pool holding the whole budget), or one
// that cannot accept the device-wide synchronisation that cudaMalloc and
// cudaFree can cause while other streams are running.  They pass their own
// input and output buffers; the scratch lives in a static array that the
// driver places in device memory when the library is loaded.
#include <string.h>

#include <mutex>

#include "internal.cuh"

namespace thoi {

constexpr size_t NOALLOC_SCRATCH_BYTES = 1u << 20;  // 1 MiB per device, held until exit
constexpr int NOALLOC_MAX_TOP_M = 16;
constexpr int NOALLOC_MAX_PARTS = 512;

// Layout inside the scratch array (byte offsets, all 256-aligned).
constexpr size_t NA_STATUS = 0;
constexpr size_t NA_BINOM = 256;
constexpr size_t NA_R64 = NA_BINOM + ((size_t)NB * NB * 8 + 255) / 256 * 256;
constexpr size_t NA_R32 = NA_R64 + (size_t)THOI_MAX_N * THOI_MAX_N * 8;
constexpr size_t NA_LS = NA_R32 + (size_t)THOI_MAX_N * THOI_MAX_N * 4;
constexpr size_t NA_PART = NA_LS + 512;
constexpr size_t NA_TOP = NA_PART + ((size_t)NOALLOC_MAX_PARTS * sizeof(PartRec) + 255) / 256 * 256;
constexpr size_t NA_END = NA_TOP + (size_t)NOALLOC_MAX_PARTS * 2 * NOALLOC_MAX_TOP_M * sizeof(TopEnt);
static_assert(NA_END <= NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the static array");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Pascal's triangle into the scratch binomial table (one thread; 4225 adds).
// The table never changes, so it is filled once per device (below).
__global__ void k_fill_binom(unsigned long long* b) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int n = 0; n < NB; n++) {
    b[n * NB] = 1ull;
    for (int m = 1; m < NB; m++) b[n * NB + m] = n == 0 ? 0ull : b[(n - 1) * NB + m - 1] + b[(n - 1) * NB + m];
  }
}

// Device address of the scratch array per device.  In host code the symbol
// name is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress with the device current.  The first call on a device
// also fills the binomial table in the array and waits for it, under the
// same lock, so later calls find it complete.
constexpr int NOALLOC_MAX_DEVICES = 64;
static void* g_scratch_addr[NOALLOC_MAX_DEVICES];
static std::mutex g_scratch_mu;

static cudaError_t scratch_for_device(int dev, cudaStream_t s, unsigned char** out) {
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    k_fill_binom<<<1, 1, 0, s>>>((unsigned long long*)((unsigned char*)p + NA_BINOM));
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = (unsigned char*)g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace thoi

using namespace thoi;

// Device (or managed) memory of device `dev`: the kernels run on the
// current device and must not touch another GPU's memory.
static bool dev_ptr(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) &&
         at.device == dev;
}

extern "C" thoi_status thoi_order_record_noalloc(const double* Sigma, int64_t N, int32_t k,
                                                 int32_t top_m, thoi_order_record* rec_out,
                                                 thoi_top_entry* top_out, void* stream) {
  if (N > THOI_MAX_N || top_m > NOALLOC_MAX_TOP_M) return THOI_ERR_TOO_LARGE;
  if (!Sigma || !rec_out || N < 1 || k < 1 || k > N || top_m < 0) return THOI_ERR_INVALID_ARG;
  if (top_m > 0 && !top_out) return THOI_ERR_INVALID_ARG;
  int dev = 0, num_sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return THOI_ERR_CUDA;
  if (!dev_ptr(Sigma, dev) || !dev_ptr(rec_out, dev) || (top_m > 0 && !dev_ptr(top_out, dev)))
    return THOI_ERR_INVALID_ARG;
  // C(N, k) by Pascal's rule on one row (no allocation); one launch indexes
  // its nplets with 32-bit offsets
  unsigned long long row[THOI_MAX_N + 1] = {1ull};
  for (int n = 1; n <= N; n++)
    for (int m = n; m >= 1; m--) row[m] += row[m - 1];
  const unsigned long long n_nplets = row[k];
  if (n_nplets > 0xffffffffull) return THOI_ERR_TOO_LARGE;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* base = nullptr;
  if (scratch_for_device(dev, s, &base) != cudaSuccess) return THOI_ERR_CUDA;
  int* status = (int*)(base + NA_STATUS);
  unsigned long long* binom = (unsigned long long*)(base + NA_BINOM);
  double* R64 = (double*)(base + NA_R64);
  float* R32 = (float*)(base + NA_R32);
  double* ls = (double*)(base + NA_LS);
  PartRec* part = (PartRec*)(base + NA_PART);
  TopEnt* top = (TopEnt*)(base + NA_TOP);
  if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return THOI_ERR_CUDA;
  // the status word must start at zero; everything else is fully rewritten
  // (the binomial table was filled by the device's first call)
  if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return THOI_ERR_CUDA;
  if (launch_normalise(Sigma, nullptr, (int)N, R64, R32, ls, nullptr, status, s) != cudaSuccess)
    return THOI_ERR_CUDA;
  NpletArgs a;
  memset(&a, 0, sizeof a);
  a.N = (int)N;
  a.k = k;
  a.R32 = R32;
  a.R64 = R64;
  a.ls = ls;
  a.binom = binom;
  a.rank_begin = 0;
  a.rank_end = n_nplets;
  a.id_base = 0;
  a.cmb.h_c = 0.5 * k * 2.8378770664093454835606594728112;
  a.cmb.tc_c = 0.0;
  a.cmb.dtc_c = 0.0;
  a.cmb.top = THOI_O;
  a.cmb.pad = 0;
  a.mode = 1;
  a.part = part;
  a.part_top = top;
  a.top_m = top_m;
  a.status = status;
  int grid = 0;
  const int cap = num_sms * 2 < NOALLOC_MAX_PARTS ? num_sms * 2 : NOALLOC_MAX_PARTS;
  if (launch_nplet_f64(a, num_sms, s, &grid, cap) != cudaSuccess) return THOI_ERR_CUDA;
  MergeDescs D;
  memset(&D, 0, sizeof D);
  D.d[0].p32_off = 0;
  D.d[0].g32 = grid;
  D.d[0].p64_off = 0;
  D.d[0].g64 = 0;
  D.d[0].k = k;
  D.d[0].cmb = a.cmb;
  D.d[0].refactored = nullptr;
  if (launch_merge(D, 1, part, top, part, top, top_m, rec_out, (TopEnt*)top_out, s) != cudaSuccess)
    return THOI_ERR_CUDA;
  int h = 0;
  if (cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return THOI_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return THOI_ERR_CUDA;
  if (h & ST_BAD_ARG) return THOI_ERR_INVALID_ARG;
  if (h & ST_NOT_PD) return THOI_ERR_NOT_PD;
  return THOI_OK;
}
