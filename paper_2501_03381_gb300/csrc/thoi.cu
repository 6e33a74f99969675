// Host side of the C ABI declared in include/thoi.h: validation, context
// and workspace ownership, the per-order launch plan, the FP64 re-factor and
// the merge, and the status word.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace thoi;

namespace thoi {
cudaError_t launch_nplet_f32(const NpletArgs& a, const Shape& sh, int num_sms, cudaStream_t s,
                             int* grid_out, int max_blocks);
}  // namespace thoi

#define CK(x)                                        \
  do {                                               \
    cudaError_t e_ = (x);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_);     \
  } while (0)

static thread_local char g_last_cuda[256];

static thoi_status cuda_fail(cudaError_t e) {
  snprintf(g_last_cuda, sizeof g_last_cuda, "%s", cudaGetErrorString(e));
  // reset the thread's last-error state, so that a failed call which leaves
  // the context usable (an allocation refused) is not reported again by the
  // cudaGetLastError check after a later launch
  cudaGetLastError();
  if (e == cudaErrorMemoryAllocation) return THOI_ERR_OOM;
  return THOI_ERR_CUDA;
}

// ------------------------------------------------------------------ context
struct thoi_ctx {
  int device = 0;
  int num_sms = 0;
  char gpu_name[256] = {0};
  int N = 0;
  long long T = 0;
  long long T_bias = 0;
  int has_ranks = 0;
  thoi_options opt;
  // tables (device)
  double* sig64 = nullptr;   // N x N covariance (FP64)
  float* sig32 = nullptr;    // N x N covariance the FP32 path starts from
  double* R64 = nullptr;
  float* R32 = nullptr;
  double* ls = nullptr;
  unsigned long long* binom = nullptr;  // NB x NB
  int* ranks = nullptr;      // T x N
  int* status = nullptr;
  int* h_cancel = nullptr;   // mapped host flag
  int* d_cancel = nullptr;
  // workspace
  unsigned long long* flag_ids = nullptr;
  size_t flag_cap = 0;
  // FP32 path: consecutive orders alternate between two re-factor lists (and
  // their FP64 basis arrays), so that the FP64 re-factor of order k runs on
  // a second stream while the FP32 kernel of order k + 1 fills the other list
  unsigned long long* flag_ids2 = nullptr;
  size_t flag_cap2 = 0;
  double* b64_2 = nullptr;
  size_t b64_2_cap = 0;
  cudaStream_t s2 = nullptr;
  std::vector<cudaEvent_t> sev;  // per-slot "list filled" and "re-factor done" events
  // group objectives (first context of a group): streams on which the
  // datasets' passes run side by side, their join events and a fork event
  std::vector<cudaStream_t> gs;
  std::vector<cudaEvent_t> gev;
  unsigned long long* flag_counts = nullptr;  // [MAX_SLOTS]
  unsigned long long* work_ctr = nullptr;     // [MAX_SLOTS] prefix-kernel work counters
  PartRec* part32 = nullptr;
  TopEnt* top32 = nullptr;
  size_t part32_cap = 0;      // blocks
  PartRec* part64 = nullptr;
  TopEnt* top64 = nullptr;
  size_t part64_cap = 0;
  int part_top_m = 0;
  unsigned char* rec_buf = nullptr;  // device staging for records
  size_t rec_cap = 0;
  double* gpart = nullptr;    // gradient partials
  size_t gpart_cap = 0;       // doubles
  float* basis = nullptr;     // FP32 path: three basis values per nplet of one piece
  size_t basis_cap = 0;       // floats
  double* b64 = nullptr;      // FP64 basis values (FP64 path pieces, re-factor list)
  size_t b64_cap = 0;         // doubles
  float* seed_thr = nullptr;  // starting top-M thresholds of the streaming reduction (2 floats)
  // fused records: candidate counters and threshold keys per order slot, then
  // the candidate list (ids, and three FP32 basis arrays of fz_cap entries)
  unsigned char* fz = nullptr;
  unsigned long long fz_cap = 0;
  int fz_used = 0;  // the last measure pass used fused records
  // radix-select workspaces: [0] the main stream, [1] the re-factor stream
  unsigned char* sel_ws = nullptr;
  // profiling: event pairs around launches, by class (0 nplet, 1 refactor, 2 merge, 3 reduce)
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_class;
  int ev_used = 0;
  // autotuner: a shape forced for the duration of a timing run
  int force_shape_valid = 0;
  Shape force_shape;
  unsigned long long serial = 0;  // unique per context (keys the batch graph cache)
  int top_meas = THOI_O;          // measure ranked by the top-M lists
  int out_sel = 0;                // per-nplet output: 0 = five measures, m + 1 = measure m alone
  // group objectives (held by the first context of a group)
  double* grp = nullptr;          // per-dataset values of one piece, then the basis of the objective
  size_t grp_cap = 0;             // doubles
  unsigned char* grp_meta = nullptr;  // dataset descriptors, status word, re-factor counters
  size_t grp_meta_cap = 0;
};

// ------------------------------------------------------------------ occupancy cache
namespace thoi {
static std::mutex g_occ_mu;
static std::map<std::pair<const void*, size_t>, int> g_occ;   // (kernel, smem, device) -> blocks/SM
static std::map<std::pair<const void*, int>, size_t> g_attr;  // (kernel, device) -> smem limit set
cudaError_t occupancy_cached(const void* fn, int block, size_t smem, int* occ) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_occ_mu);
  // the kernel's dynamic shared-memory limit only ever grows, so every size
  // launched before stays valid
  const std::pair<const void*, int> akey(fn, dev);
  auto at = g_attr.find(akey);
  if (at == g_attr.end() || at->second < smem) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    g_attr[akey] = smem;
  }
  const std::pair<const void*, size_t> key(fn, smem * 64 + (size_t)dev);
  auto it = g_occ.find(key);
  if (it != g_occ.end()) {
    *occ = it->second;
    return cudaSuccess;
  }
  int o = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, block, smem);
  if (e != cudaSuccess) return e;
  if (o < 1) o = 1;
  g_occ[key] = o;
  *occ = o;
  return cudaSuccess;
}
}  // namespace thoi

// ------------------------------------------------------------------ autotune cache
// Process-wide: (GPU name, SM count, order, mask width, use) -> launch shape.
// Two uses per order: records reduced in place (nothing stored per nplet),
// and per-nplet output (every value stored at its rank, where the dense
// kernels' coalesced stores can outweigh the prefix kernels' fewer FLOPs).
static std::mutex g_tune_mu;
static std::map<std::string, Shape> g_tune;
// the batched kernel's per-order chunks, tuned on a batch (kept apart from
// the single-dataset shapes, which the JSON cache holds)
static std::map<std::string, Shape> g_tune_batch;
static unsigned long long g_tune_gen = 0;  // bumped whenever g_tune changes

static std::string tune_key(const char* gpu, int sms, int k, int wide, int out = 0) {
  char b[320];
  snprintf(b, sizeof b, "%s|%d|%d|%d|%d", gpu, sms, k, wide, out);
  return b;
}

// out: the launch stores every nplet's measures (per-nplet output)
static Shape shape_for(const thoi_ctx* c, int k, int out) {
  if (c->force_shape_valid) return c->force_shape;
  if (c->opt.autotune) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(tune_key(c->gpu_name, c->num_sms, k, c->N > 32, out));
    if (it != g_tune.end()) return it->second;
  }
  return default_shape(k);
}

static thoi_status prof_begin(thoi_ctx* c, cudaStream_t s, int cls) {
  if (!c->opt.profile) return THOI_OK;
  while ((int)c->ev.size() < 2 * (c->ev_used + 1)) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    c->ev.push_back(e);
  }
  if ((int)c->ev_class.size() < c->ev_used + 1) c->ev_class.resize(c->ev_used + 1);
  c->ev_class[c->ev_used] = cls;
  CK(cudaEventRecord(c->ev[2 * c->ev_used], s));
  return THOI_OK;
}
static thoi_status prof_end(thoi_ctx* c, cudaStream_t s) {
  if (!c->opt.profile) return THOI_OK;
  CK(cudaEventRecord(c->ev[2 * c->ev_used + 1], s));
  c->ev_used++;
  return THOI_OK;
}

static void free_ptr(void* p) {
  if (p) cudaFree(p);
}

template <typename T>
static thoi_status grow(T** p, size_t* cap, size_t need_elems) {
  if (*cap >= need_elems && *p) return THOI_OK;
  free_ptr(*p);
  *p = nullptr;
  *cap = 0;
  if (need_elems == 0) return THOI_OK;
  CK(cudaMalloc((void**)p, need_elems * sizeof(T)));
  *cap = need_elems;
  return THOI_OK;
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------------------ host math
static uint64_t binom_host(int n, int k) {
  static uint64_t tab[NB][NB];
  static std::once_flag once;
  std::call_once(once, [] {
    for (int a = 0; a < NB; a++) {
      tab[a][0] = 1;
      for (int b = 1; b < NB; b++) tab[a][b] = a == 0 ? 0 : tab[a - 1][b - 1] + tab[a - 1][b];
    }
  });
  if (n < 0 || k < 0 || n >= NB || k >= NB) return 0;
  return tab[n][k];
}

// Digamma by upward recurrence to x >= 8 and the Stirling-type series.
static double digamma_host(double x) {
  double acc = 0.0;
  for (; x < 8.0; x += 1.0) acc -= 1.0 / x;
  const double x2 = 1.0 / (x * x);
  const double series =
      x2 * (1.0 / 12 - x2 * (1.0 / 120 - x2 * (1.0 / 252 - x2 * (1.0 / 240 - x2 * (1.0 / 132)))));
  return acc + log(x) - 0.5 / x - series;
}

// Gaussian entropy bias of m variables from T samples (Supp. eq.
// bias_corrector read with 1/2 on the digamma sum).
static double eta_host(int m, long long T) {
  if (m <= 0) return 0.0;
  double s = m * log(2.0 / (double)(T - 1));
  for (int j = 1; j <= m; j++) s += digamma_host(0.5 * (double)(T - j));
  return 0.5 * s;
}

static Combine combine_for(const thoi_ctx* c, int k) {
  const double LOG2PIE = 2.8378770664093454835606594728112;
  Combine cb;
  cb.h_c = 0.5 * k * LOG2PIE;
  cb.tc_c = 0.0;
  cb.dtc_c = 0.0;
  cb.top = c->top_meas;
  cb.pad = 0;
  if (c->opt.bias_correct && c->T_bias > k + 1) {
    const double ek = eta_host(k, c->T_bias), e1 = eta_host(1, c->T_bias),
                 ekm = eta_host(k - 1, c->T_bias);
    cb.h_c -= ek;
    cb.tc_c = -k * e1 + ek;
    cb.dtc_c = (k - 1) * ek - k * ekm;
  }
  return cb;
}

// ------------------------------------------------------------------ API: misc
extern "C" void thoi_default_options(thoi_options* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->precision = THOI_F32_FIX64;
  o->pivot_tau = 1e-2f;
  o->trace_tau = 100.0f;
  o->bias_correct = 0;
  o->top_m = 256;
  o->out_f64 = -1;
  o->sigma32_source = THOI_SIGMA32_FROM_F64;
  o->autotune = 1;
  o->flag_capacity = 0;
  o->profile = 0;
  o->records_mode = THOI_RECORDS_AUTO;
}

extern "C" const char* thoi_status_string(thoi_status s) {
  switch (s) {
    case THOI_OK: return "ok";
    case THOI_ERR_INVALID_ARG: return "invalid argument";
    case THOI_ERR_NONFINITE_INPUT: return "input holds NaN or Inf";
    case THOI_ERR_TOO_LARGE: return "size beyond a documented limit";
    case THOI_ERR_NOT_PD: return "a nplet is not positive definite";
    case THOI_ERR_OOM: return "device allocation failed";
    case THOI_ERR_CUDA: return g_last_cuda[0] ? g_last_cuda : "CUDA error";
    case THOI_ERR_TIMEOUT: return "bounded device wait gave up";
    case THOI_ERR_CANCELLED: return "cancelled";
    case THOI_ERR_WORKSPACE: return "re-factor list overflow";
  }
  return "unknown status";
}

extern "C" uint64_t thoi_count(int64_t N, const int32_t* orders, int32_t n_orders) {
  if (N < 1 || N > THOI_MAX_N || !orders || n_orders < 1) return 0;
  uint64_t s = 0;
  for (int i = 0; i < n_orders; i++) s += binom_host((int)N, orders[i]);
  return s;
}

extern "C" size_t thoi_records_bytes(int32_t n_orders, int32_t top_m) {
  if (n_orders < 0 || top_m < 0) return 0;
  return (size_t)n_orders * sizeof(thoi_order_record) +
         (size_t)n_orders * 2 * (size_t)top_m * sizeof(thoi_top_entry);
}

static bool orders_ok(int N, const int32_t* orders, int32_t n_orders) {
  if (!orders || n_orders < 1 || n_orders > MAX_SLOTS) return false;
  for (int i = 0; i < n_orders; i++)
    if (orders[i] < 1 || orders[i] > N) return false;
  return true;
}

// Host unrank: the same combinatorial number system as the device code.
extern "C" thoi_status thoi_unrank(int64_t N, const int32_t* orders, int32_t n_orders, uint64_t id,
                                   int32_t* idx_out, int32_t* k_out) {
  if (N < 1 || N > THOI_MAX_N || !orders_ok((int)N, orders, n_orders) || !idx_out)
    return THOI_ERR_INVALID_ARG;
  for (int s = 0; s < n_orders; s++) {
    const uint64_t c = binom_host((int)N, orders[s]);
    if (id < c) {
      const int k = orders[s];
      uint64_t rr = c - 1 - id;
      int d = (int)N - 1;
      for (int i = 0; i < k; i++) {
        const int m = k - i;
        while (binom_host(d, m) > rr) d--;
        rr -= binom_host(d, m);
        idx_out[i] = (int32_t)(N - 1 - d);
        d--;
      }
      if (k_out) *k_out = k;
      return THOI_OK;
    }
    id -= c;
  }
  return THOI_ERR_INVALID_ARG;
}

extern "C" thoi_status thoi_unrank_device(int64_t N, const int32_t* orders, int32_t n_orders,
                                          const uint64_t* ids, int64_t n, int32_t kmax,
                                          int8_t* idx_out, void* stream) {
  if (N < 1 || N > THOI_MAX_N || !orders_ok((int)N, orders, n_orders) || n < 0 || !ids ||
      !idx_out)
    return THOI_ERR_INVALID_ARG;
  for (int i = 0; i < n_orders; i++)
    if (orders[i] > kmax) return THOI_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<unsigned long long> hb(NB * NB), offs(n_orders + 1);
  for (int a = 0; a < NB; a++)
    for (int b = 0; b < NB; b++) hb[a * NB + b] = binom_host(a, b);
  offs[0] = 0;
  for (int i = 0; i < n_orders; i++) offs[i + 1] = offs[i] + binom_host((int)N, orders[i]);
  unsigned long long *d_b = nullptr, *d_o = nullptr;
  int* d_ord = nullptr;
  thoi_status st = THOI_OK;
  cudaError_t e = cudaMalloc(&d_b, hb.size() * 8);
  if (e == cudaSuccess) e = cudaMalloc(&d_o, offs.size() * 8);
  if (e == cudaSuccess) e = cudaMalloc(&d_ord, n_orders * 4);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_b, hb.data(), hb.size() * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_o, offs.data(), offs.size() * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_ord, orders, n_orders * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = launch_unrank_ids((int)N, d_ord, d_o, n_orders, d_b, (const unsigned long long*)ids, n, kmax,
                          idx_out, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) st = cuda_fail(e);
  free_ptr(d_b);
  free_ptr(d_o);
  free_ptr(d_ord);
  return st;
}

extern "C" int64_t thoi_n(const thoi_ctx* c) { return c ? c->N : 0; }

extern "C" thoi_status thoi_set_cancel(thoi_ctx* c, int32_t flag) {
  if (!c || !c->h_cancel) return THOI_ERR_INVALID_ARG;
  *(volatile int*)c->h_cancel = flag ? 1 : 0;
  return THOI_OK;
}

static void batch_forget(unsigned long long serial);
static unsigned long long next_serial();

extern "C" void thoi_destroy(thoi_ctx* c) {
  if (!c) return;
  batch_forget(c->serial);
  free_ptr(c->sig64);
  free_ptr(c->sig32);
  free_ptr(c->R64);
  free_ptr(c->R32);
  free_ptr(c->ls);
  free_ptr(c->binom);
  free_ptr(c->ranks);
  free_ptr(c->status);
  if (c->h_cancel) cudaFreeHost(c->h_cancel);
  for (auto e : c->ev) cudaEventDestroy(e);
  free_ptr(c->flag_ids);
  free_ptr(c->flag_ids2);
  free_ptr(c->b64_2);
  for (auto e : c->sev) cudaEventDestroy(e);
  if (c->s2) cudaStreamDestroy(c->s2);
  for (auto e : c->gev) cudaEventDestroy(e);
  for (auto q : c->gs) cudaStreamDestroy(q);
  free_ptr(c->flag_counts);
  free_ptr(c->work_ctr);
  free_ptr(c->part32);
  free_ptr(c->top32);
  free_ptr(c->part64);
  free_ptr(c->top64);
  free_ptr(c->rec_buf);
  free_ptr(c->gpart);
  free_ptr(c->basis);
  free_ptr(c->b64);
  free_ptr(c->seed_thr);
  free_ptr(c->sel_ws);
  free_ptr(c->fz);
  free_ptr(c->grp);
  free_ptr(c->grp_meta);
  delete c;
}

// ------------------------------------------------------------------ API: create
static thoi_status ctx_common(thoi_ctx* c, int N, const thoi_options* opt) {
  if (opt) c->opt = *opt;
  else thoi_default_options(&c->opt);
  if (c->opt.out_f64 < 0) c->opt.out_f64 = c->opt.precision == THOI_F64 ? 1 : 0;
  if (c->opt.precision != THOI_F32_FIX64 && c->opt.precision != THOI_F64) return THOI_ERR_INVALID_ARG;
  if (c->opt.top_m < 0 || c->opt.top_m > THOI_MAX_TOP_M) return THOI_ERR_INVALID_ARG;
  if (!(c->opt.pivot_tau >= 0.0f) || !(c->opt.trace_tau > 0.0f)) return THOI_ERR_INVALID_ARG;
  if (c->opt.sigma32_source != THOI_SIGMA32_TENSORCORE &&
      c->opt.sigma32_source != THOI_SIGMA32_FROM_F64)
    return THOI_ERR_INVALID_ARG;
  if (c->opt.records_mode < THOI_RECORDS_AUTO || c->opt.records_mode > THOI_RECORDS_STORED)
    return THOI_ERR_INVALID_ARG;
  c->N = N;
  c->serial = next_serial();
  CK(cudaGetDevice(&c->device));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, c->device));
  c->num_sms = prop.multiProcessorCount;
  snprintf(c->gpu_name, sizeof c->gpu_name, "%s", prop.name);
  CK(cudaMalloc(&c->sig64, (size_t)N * N * 8));
  CK(cudaMalloc(&c->sig32, (size_t)N * N * 4));
  CK(cudaMalloc(&c->R64, (size_t)N * N * 8));
  CK(cudaMalloc(&c->R32, (size_t)N * N * 4));
  CK(cudaMalloc(&c->ls, (size_t)N * 8));
  CK(cudaMalloc(&c->binom, (size_t)NB * NB * 8));
  CK(cudaMalloc(&c->status, sizeof(int)));
  CK(cudaMalloc(&c->flag_counts, MAX_SLOTS * sizeof(unsigned long long)));
  CK(cudaMalloc(&c->work_ctr, MAX_SLOTS * sizeof(unsigned long long)));
  CK(cudaMalloc(&c->seed_thr, 2 * sizeof(float)));
  CK(cudaHostAlloc(&c->h_cancel, sizeof(int), cudaHostAllocMapped));
  *c->h_cancel = 0;
  CK(cudaHostGetDevicePointer((void**)&c->d_cancel, c->h_cancel, 0));
  std::vector<unsigned long long> hb(NB * NB);
  for (int a = 0; a < NB; a++)
    for (int b = 0; b < NB; b++) hb[a * NB + b] = binom_host(a, b);
  CK(cudaMemcpy(c->binom, hb.data(), hb.size() * 8, cudaMemcpyHostToDevice));
  return THOI_OK;
}

static thoi_status read_status(thoi_ctx* c, cudaStream_t s, int* out) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, c->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *out = h;
  return THOI_OK;
}

extern "C" thoi_status thoi_create(thoi_ctx** out, const void* X, int64_t T, int64_t N, int64_t ld,
                                   int32_t dtype, const thoi_options* opt, void* stream) {
  if (!out || !X) return THOI_ERR_INVALID_ARG;
  *out = nullptr;
  if (N > THOI_MAX_N) return THOI_ERR_TOO_LARGE;
  if (N < 2 || T < N + 1 || ld < N || (dtype != THOI_DTYPE_F32 && dtype != THOI_DTYPE_F64))
    return THOI_ERR_INVALID_ARG;
  if (T > (1ll << 24)) return THOI_ERR_TOO_LARGE;
  cudaStream_t s = (cudaStream_t)stream;
  thoi_ctx* c = new thoi_ctx();
  thoi_status st = ctx_common(c, (int)N, opt);
  if (st != THOI_OK) { thoi_destroy(c); return st; }
  c->T = T;
  c->T_bias = T;
  c->has_ranks = 1;
  const size_t esz = dtype == THOI_DTYPE_F64 ? 8 : 4;
  const bool dev = is_device_ptr(X);
  void* dX = nullptr;
  const void* Xuse = X;
  CopulaWs w;
  memset(&w, 0, sizeof w);
  CopulaWsSizes z;
  copula_ws_sizes(T, (int)N, &z);
  const int tc = c->opt.sigma32_source == THOI_SIGMA32_TENSORCORE;
  cudaError_t e = cudaSuccess;
#define TRY(x) if (e == cudaSuccess) e = (x)
  if (!dev) {
    TRY(cudaMalloc(&dX, (size_t)T * ld * esz));
    TRY(cudaMemcpyAsync(dX, X, (size_t)T * ld * esz, cudaMemcpyHostToDevice, s));
    Xuse = dX;
  }
  TRY(cudaMalloc(&c->ranks, (size_t)T * N * 4));
  w.rank = c->ranks;
  TRY(cudaMalloc(&w.ztab, (size_t)T * 8));
  TRY(cudaMalloc(&w.Z, (size_t)T * N * 8));
  TRY(cudaMalloc(&w.mu, (size_t)N * 8));
  w.sig64 = c->sig64;
  if (tc) {
    const size_t nz = (size_t)z.Np * z.Tp * 2;
    TRY(cudaMalloc(&w.zh, nz));
    TRY(cudaMalloc(&w.zm, nz));
    TRY(cudaMalloc(&w.zl, nz));
    TRY(cudaMalloc(&w.part, (size_t)z.n_chunks * z.Np * z.Np * 8));
    TRY(cudaMalloc(&w.sig32acc, (size_t)N * N * 8));
  }
  TRY(cudaMemsetAsync(c->status, 0, sizeof(int), s));
  TRY(launch_copula(Xuse, dtype, T, (int)N, ld, w, tc, c->status, s));
  TRY(launch_normalise(c->sig64, tc ? w.sig32acc : nullptr, (int)N, c->R64, c->R32, c->ls, c->sig32,
                       c->status, s));
  TRY(cudaStreamSynchronize(s));
#undef TRY
  free_ptr(dX);
  free_ptr(w.ztab);
  free_ptr(w.Z);
  free_ptr(w.mu);
  free_ptr(w.zh);
  free_ptr(w.zm);
  free_ptr(w.zl);
  free_ptr(w.part);
  free_ptr(w.sig32acc);
  if (e != cudaSuccess) { thoi_destroy(c); return cuda_fail(e); }
  int hs = 0;
  st = read_status(c, s, &hs);
  if (st != THOI_OK) { thoi_destroy(c); return st; }
  if (hs & ST_NONFINITE) { thoi_destroy(c); return THOI_ERR_NONFINITE_INPUT; }
  if (hs & ST_BAD_ARG) { thoi_destroy(c); return THOI_ERR_INVALID_ARG; }
  *out = c;
  return THOI_OK;
}

extern "C" thoi_status thoi_create_from_cov(thoi_ctx** out, const double* Sigma, int64_t N,
                                            int64_t T_for_bias, const thoi_options* opt,
                                            void* stream) {
  if (!out || !Sigma) return THOI_ERR_INVALID_ARG;
  *out = nullptr;
  if (N > THOI_MAX_N) return THOI_ERR_TOO_LARGE;
  if (N < 1) return THOI_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  thoi_ctx* c = new thoi_ctx();
  thoi_status st = ctx_common(c, (int)N, opt);
  if (st != THOI_OK) { thoi_destroy(c); return st; }
  c->T = 0;
  c->T_bias = T_for_bias;
  if (c->opt.bias_correct && T_for_bias < N + 2) { thoi_destroy(c); return THOI_ERR_INVALID_ARG; }
  cudaError_t e = cudaMemcpyAsync(c->sig64, Sigma, (size_t)N * N * 8, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(int), s);
  if (e == cudaSuccess)
    e = launch_normalise(c->sig64, nullptr, (int)N, c->R64, c->R32, c->ls, c->sig32, c->status, s);
  if (e != cudaSuccess) { thoi_destroy(c); return cuda_fail(e); }
  int hs = 0;
  st = read_status(c, s, &hs);
  if (st != THOI_OK) { thoi_destroy(c); return st; }
  if (hs & ST_BAD_ARG) { thoi_destroy(c); return THOI_ERR_INVALID_ARG; }
  *out = c;
  return THOI_OK;
}

extern "C" thoi_status thoi_get_cov(thoi_ctx* c, double* S64, float* S32, void* stream) {
  if (!c) return THOI_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)c->N * c->N;
  if (S64) CK(cudaMemcpyAsync(S64, c->sig64, n * 8, cudaMemcpyDefault, s));
  if (S32) CK(cudaMemcpyAsync(S32, c->sig32, n * 4, cudaMemcpyDefault, s));
  CK(cudaStreamSynchronize(s));
  return THOI_OK;
}

extern "C" thoi_status thoi_get_ranks(thoi_ctx* c, int32_t* ranks, void* stream) {
  if (!c || !ranks || !c->has_ranks) return THOI_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(ranks, c->ranks, (size_t)c->T * c->N * 4, cudaMemcpyDefault, s));
  CK(cudaStreamSynchronize(s));
  return THOI_OK;
}

// ------------------------------------------------------------------ API: measures
namespace {

struct SlotRange {
  int k;
  unsigned long long off;     // global id of rank 0
  unsigned long long r0, r1;  // rank range inside [id_begin, id_end)
};

constexpr int MAX_BLOCKS_PER_SM_RED = 8;   // cap for reduction launches (partials per block)
constexpr int MAX_BLOCKS_PER_SM_OUT = 8;
constexpr int REFACTOR_BLOCKS_PER_SM = 2;
constexpr int LIST_RED_BLOCKS = 16;  // blocks of the re-factor list's reduction
constexpr unsigned long long LAUNCH_SPLIT = 0xffffffffull;  // ranks per launch (u32 local ids)
constexpr unsigned long long PIECE = 1ull << 28;  // FP32 records path: nplets per basis piece
constexpr unsigned long long FUSE_MIN_N = 1ull << 20;  // automatic fused records from this size
const int FUSE_CAND_BLOCKS = cand_partials(FUSE_NSEG);  // candidate-reduction partials per slot
// head of the fused workspace: MAX_SLOTS x FUSE_NSEG segment counters (8 KB),
// then MAX_SLOTS x 10 threshold keys (2.5 KB)
constexpr size_t FZ_COUNTS = (size_t)MAX_SLOTS * FUSE_NSEG * 8;
constexpr size_t FZ_HEAD = FZ_COUNTS + 2560 + 512;

// Elements between the three basis arrays: the piece length rounded up to a
// multiple of 64, so that every array is 256-byte aligned.
unsigned long long basis_stride(unsigned long long max_slot_nplets) {
  const unsigned long long piece = max_slot_nplets < PIECE ? max_slot_nplets : PIECE;
  return ((piece > 0 ? piece : 1) + 63) / 64 * 64;
}

}  // namespace

static thoi_status plan_slots(const thoi_ctx* c, const int32_t* orders, int32_t n_orders,
                              uint64_t id_begin, uint64_t* id_end, std::vector<SlotRange>* slots) {
  const uint64_t total = thoi_count(c->N, orders, n_orders);
  if (*id_end == UINT64_MAX) *id_end = total;
  if (id_begin > *id_end || *id_end > total) return THOI_ERR_INVALID_ARG;
  unsigned long long off = 0;
  slots->clear();
  for (int s = 0; s < n_orders; s++) {
    const unsigned long long cnt = binom_host(c->N, orders[s]);
    SlotRange r;
    r.k = orders[s];
    r.off = off;
    const unsigned long long a = id_begin > off ? id_begin - off : 0;
    const unsigned long long b = *id_end > off ? (*id_end - off < cnt ? *id_end - off : cnt) : 0;
    r.r0 = a < cnt ? a : cnt;
    r.r1 = b > r.r0 ? b : r.r0;
    slots->push_back(r);
    off += cnt;
  }
  return THOI_OK;
}

static thoi_status ensure_flag_ws(thoi_ctx* c, unsigned long long max_slot_nplets) {
  size_t need = c->opt.flag_capacity;
  if (need == 0) {
    // automatic: 1/16 of the largest order, at least 1M, at most 64M entries
    unsigned long long a = max_slot_nplets / 16 + 1;
    if (a < (1ull << 20)) a = 1ull << 20;
    if (a > (64ull << 20)) a = 64ull << 20;
    if (a > max_slot_nplets) a = max_slot_nplets > 0 ? max_slot_nplets : 1;
    need = (size_t)a;
  }
  thoi_status st = grow(&c->flag_ids, &c->flag_cap, need);
  if (st != THOI_OK) return st;
  return grow(&c->flag_ids2, &c->flag_cap2, c->flag_cap);
}

// The second stream and the events of the overlapped FP64 re-factor.
static thoi_status ensure_overlap(thoi_ctx* c, int n_slots) {
  if (!c->s2) CK(cudaStreamCreateWithFlags(&c->s2, cudaStreamNonBlocking));
  while ((int)c->sev.size() < 2 * n_slots + 1) {
    cudaEvent_t e;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    c->sev.push_back(e);
  }
  return THOI_OK;
}

// si >= 0: the request's order slot (the prefix-shared kernels take their
// work from that slot's counter, zeroed with the request)
static NpletArgs base_args(thoi_ctx* c, const SlotRange& r, int si = -1) {
  NpletArgs a;
  memset(&a, 0, sizeof a);
  if (si >= 0) a.work_counter = c->work_ctr + si;
  a.N = c->N;
  a.k = r.k;
  a.R32 = c->R32;
  a.R64 = c->R64;
  a.ls = c->ls;
  a.binom = c->binom;
  a.rank_begin = r.r0;
  a.rank_end = r.r1;
  a.id_base = r.off;
  a.cmb = combine_for(c, r.k);
  a.out_sel = c->out_sel;
  a.tau_piv = c->opt.pivot_tau;
  a.tau_tr = c->opt.trace_tau;
  a.status = c->status;
  a.cancel = c->d_cancel;
  a.flag_ids = c->flag_ids;
  a.flag_cap = c->flag_cap;
  return a;
}

static thoi_status finish_status(thoi_ctx* c, cudaStream_t s, int n_slots, thoi_stats* stats,
                                 uint64_t nplets, int launches, int* hs_out = nullptr) {
  int hs = 0;
  unsigned long long fc[MAX_SLOTS];
  CK(cudaMemcpyAsync(&hs, c->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (n_slots > 0)
    CK(cudaMemcpyAsync(fc, c->flag_counts, n_slots * 8, cudaMemcpyDeviceToHost, s));
  std::vector<unsigned long long> cc;
  if (c->fz_used && c->fz) {
    cc.resize((size_t)MAX_SLOTS * FUSE_NSEG);
    CK(cudaMemcpyAsync(cc.data(), c->fz, cc.size() * 8, cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  unsigned long long nref = 0, ncand = 0;
  for (int i = 0; i < n_slots; i++) nref += fc[i] < c->flag_cap ? fc[i] : c->flag_cap;
  for (auto x : cc) ncand += x;
  double ms[4] = {0, 0, 0, 0};
  for (int i = 0; i < c->ev_used; i++) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, c->ev[2 * i], c->ev[2 * i + 1]));
    ms[c->ev_class[i]] += t;
  }
  c->ev_used = 0;
  if (stats) {
    memset(stats, 0, sizeof *stats);
    stats->nplets = nplets;
    stats->n_refactored = nref;
    stats->n_not_pd = 0;
    stats->launches = launches;
    stats->nplet_ms = ms[0];
    stats->refactor_ms = ms[1];
    stats->merge_ms = ms[2];
    stats->reduce_ms = ms[3];
    stats->n_candidates = ncand;
  }
  if (hs_out) *hs_out = hs;
  if (hs & ST_FLAG_OVERFLOW) return THOI_ERR_WORKSPACE;
  if (hs & ST_CANCELLED) return THOI_ERR_CANCELLED;
  if (hs & ST_NOT_PD) return THOI_ERR_NOT_PD;
  return THOI_OK;
}

// Reduction partials of n32 blocks (FP32 or FP64 path) and n64 blocks (FP64
// re-factor), each with two top lists of top_m entries.
static thoi_status ensure_parts(thoi_ctx* c, size_t n32, size_t n64, int top_m) {
  if (c->part_top_m != top_m) {
    free_ptr(c->top32); c->top32 = nullptr;
    free_ptr(c->top64); c->top64 = nullptr;
    free_ptr(c->part32); c->part32 = nullptr; c->part32_cap = 0;
    free_ptr(c->part64); c->part64 = nullptr; c->part64_cap = 0;
    c->part_top_m = top_m;
  }
  size_t cap32 = c->part32_cap, cap64 = c->part64_cap;
  thoi_status st = grow(&c->part32, &c->part32_cap, n32 > 0 ? n32 : 1);
  if (st != THOI_OK) return st;
  if (c->part32_cap != cap32 || !c->top32) {
    free_ptr(c->top32);
    c->top32 = nullptr;
    if (top_m > 0) CK(cudaMalloc(&c->top32, c->part32_cap * 2 * top_m * sizeof(TopEnt)));
  }
  st = grow(&c->part64, &c->part64_cap, n64 > 0 ? n64 : 1);
  if (st != THOI_OK) return st;
  if (c->part64_cap != cap64 || !c->top64) {
    free_ptr(c->top64);
    c->top64 = nullptr;
    if (top_m > 0) CK(cudaMalloc(&c->top64, c->part64_cap * 2 * top_m * sizeof(TopEnt)));
  }
  return THOI_OK;
}

// Candidate-list entries for a fused slot of n nplets.  The sample bounds of
// the top lists pass, per side, about 6 / (samples per block) of the nplets
// (the smallest of 256 block maxima), and each extreme of the other measures
// about n / S; three times the expected count, at least 2^16, at most n.
static unsigned long long fused_cand_cap(unsigned long long n, int top_m) {
  const unsigned long long grid = top_m > 256 ? (unsigned long long)top_m : 256ull;
  unsigned long long S = grid * 128ull * (unsigned long long)fused_sample_per_thread(n, top_m);
  if (S > n) S = n;
  const double per_block = (double)S / (double)grid;
  const double expect = 2.0 * 6.0 * (double)n / (per_block > 1.0 ? per_block : 1.0) +
                        10.0 * (double)n / (double)(S > 0 ? S : 1);
  unsigned long long cap = (unsigned long long)(3.0 * expect) + (1ull << 16);
  return cap < n ? cap : n;
}

// Fused records workspace for candidate lists of up to cap entries, cut
// into FUSE_NSEG segments; every array and segment starts on a 256-byte
// boundary.
static thoi_status ensure_fused_ws(thoi_ctx* c, unsigned long long cap_need) {
  unsigned long long seg = (cap_need + FUSE_NSEG - 1) / FUSE_NSEG;
  seg = (seg + 63) / 64 * 64;
  const unsigned long long cap = seg * FUSE_NSEG;
  if (c->fz && c->fz_cap >= cap) return THOI_OK;
  free_ptr(c->fz);
  c->fz = nullptr;
  c->fz_cap = 0;
  CK(cudaMalloc(&c->fz, FZ_HEAD + (size_t)cap * 8 + (size_t)cap * 3 * 4 + cand_ws_bytes()));
  c->fz_cap = cap;
  return THOI_OK;
}
static thoi_status ensure_sel_ws(thoi_ctx* c) {
  if (c->sel_ws) return THOI_OK;
  CK(cudaMalloc(&c->sel_ws, 2 * sel_ws_bytes()));
  return THOI_OK;
}
// Kernels of one radix-select reduction: three passes and the final sort
// (with top lists), else the first pass and an empty top partial.
static int sel_kernels(int top_m) { return top_m > 0 ? 4 : 2; }
static unsigned long long* fz_counts(thoi_ctx* c) { return (unsigned long long*)c->fz; }
static unsigned* fz_keys(thoi_ctx* c) { return (unsigned*)(c->fz + FZ_COUNTS); }
static unsigned long long* fz_ids(thoi_ctx* c) { return (unsigned long long*)(c->fz + FZ_HEAD); }
static float* fz_basis(thoi_ctx* c) { return (float*)(c->fz + FZ_HEAD + (size_t)c->fz_cap * 8); }
static unsigned char* fz_ws(thoi_ctx* c) { return c->fz + FZ_HEAD + (size_t)c->fz_cap * 20; }

// Queue the whole measure pass (no synchronisation).  Used directly by the
// batched entry point, which captures it into a CUDA graph.  With `fuse`,
// per-order records of the FP32 path reduce inside the nplet kernels where
// the context's records_mode allows (see fused records in nplet_common.cuh).
static thoi_status enqueue_measures(thoi_ctx* c, const int32_t* orders, int32_t n_orders,
                                    uint64_t id_begin, uint64_t id_end, int32_t kind, void* out_dev,
                                    thoi_order_record* recs_dev, TopEnt* tops_dev,
                                    cudaStream_t s, int* launches_out, bool fuse = false,
                                    bool sel64 = false) {
  std::vector<SlotRange> slots;
  thoi_status st = plan_slots(c, orders, n_orders, id_begin, &id_end, &slots);
  if (st != THOI_OK) return st;
  const bool red = kind == THOI_RED_PER_ORDER;
  const bool f64 = c->opt.precision == THOI_F64;
  const int top_m = red ? c->opt.top_m : 0;
  int launches = 0;
  c->ev_used = 0;
  unsigned long long maxn = 0, maxn_fused = 0;
  for (auto& r : slots) maxn = (r.r1 - r.r0) > maxn ? (r.r1 - r.r0) : maxn;
  auto fused_slot = [&](const SlotRange& r) {
    const unsigned long long n = r.r1 - r.r0;
    if (!fuse || !red || f64 || c->opt.records_mode == THOI_RECORDS_STORED) return false;
    if (n == 0 || n > PIECE || r.k > 32) return false;
    return c->opt.records_mode == THOI_RECORDS_FUSED || n >= FUSE_MIN_N;
  };
  unsigned long long cand_need = 0;
  for (auto& r : slots) {
    if (!fused_slot(r)) continue;
    const unsigned long long n = r.r1 - r.r0;
    if (n > maxn_fused) maxn_fused = n;
    const unsigned long long cc = fused_cand_cap(n, c->opt.top_m);
    if (cc > cand_need) cand_need = cc;
  }
  if (maxn_fused > 0) {
    st = ensure_fused_ws(c, cand_need);
    if (st != THOI_OK) return st;
  }
  // radix-select reductions (short stored ranges, re-factor lists) on the
  // first pass of a records request; a repeat uses the streaming reductions
  const bool sel = fuse && red && c->opt.records_mode != THOI_RECORDS_STORED;
  if (sel || sel64) {
    st = ensure_sel_ws(c);
    if (st != THOI_OK) return st;
  }
  if (!f64) {
    st = ensure_flag_ws(c, maxn);
    if (st != THOI_OK) return st;
  }
  // partial buffers for the reductions: one region per launch
  const int blk_cap = c->num_sms * MAX_BLOCKS_PER_SM_RED;
  const int ref_cap = c->num_sms * REFACTOR_BLOCKS_PER_SM;
  if (red) {
    size_t n32 = 0;
    const unsigned long long split = f64 ? LAUNCH_SPLIT : PIECE;
    for (auto& r : slots) {
      const unsigned long long n = r.r1 - r.r0;
      const size_t parts = n == 0 ? 0 : (size_t)((n + split - 1) / split);
      n32 += parts * blk_cap + (fused_slot(r) ? FUSE_CAND_BLOCKS : 0);
    }
    if (!f64) {
      st = grow(&c->basis, &c->basis_cap, (size_t)3 * basis_stride(maxn));
      if (st != THOI_OK) return st;
    }
    {
      // FP64 basis scratch: pieces of the FP64 path, or the re-factor list
      const size_t need = f64 ? (size_t)3 * basis_stride(maxn)
                              : (size_t)3 * (((size_t)c->flag_cap + 63) / 64 * 64);
      st = grow(&c->b64, &c->b64_cap, need);
      if (st != THOI_OK) return st;
      if (!f64) {
        st = grow(&c->b64_2, &c->b64_2_cap, need);
        if (st != THOI_OK) return st;
      }
    }
    const size_t n64 = f64 ? 0 : slots.size() * (size_t)ref_cap;
    st = ensure_parts(c, n32, n64, top_m);
    if (st != THOI_OK) return st;
  }
  CK(cudaMemsetAsync(c->status, 0, sizeof(int), s));
  CK(cudaMemsetAsync(c->flag_counts, 0, MAX_SLOTS * sizeof(unsigned long long), s));
  CK(cudaMemsetAsync(c->work_ctr, 0, MAX_SLOTS * sizeof(unsigned long long), s));
  if (maxn_fused > 0) CK(cudaMemsetAsync(c->fz, 0, FZ_HEAD, s));  // counters and keys
  // the FP64 re-factor of each order on a second stream (FP32 path, several
  // orders): its FP64 work overlaps the next order's FP32 kernel
  const bool overlap = !f64 && slots.size() > 1;
  if (overlap) {
    st = ensure_overlap(c, (int)slots.size());
    if (st != THOI_OK) return st;
  }
  c->fz_used = maxn_fused > 0;

  MergeDescs D;
  memset(&D, 0, sizeof D);
  int p32_off = 0, p64_off = 0;
  for (size_t si = 0; si < slots.size(); si++) {
    const SlotRange& r = slots[si];
    MergeDesc& md = D.d[si];
    md.k = r.k;
    md.cmb = combine_for(c, r.k);
    md.p32_off = p32_off;
    md.p64_off = p64_off;
    md.refactored = f64 ? nullptr : c->flag_counts + si;
    const Shape sh = shape_for(c, r.k, kind == THOI_RED_NONE);
    // this order's re-factor list (the two lists alternate between orders)
    unsigned long long* const fids = (si & 1) ? c->flag_ids2 : c->flag_ids;
    double* const fb64 = (si & 1) ? c->b64_2 : c->b64;
    if (overlap && si >= 2) CK(cudaStreamWaitEvent(s, c->sev[2 * (si - 2) + 1], 0));
    if (fused_slot(r)) {
      // fused records: sample bounds, the nplet kernel reducing in place, the
      // candidate list's reduction
      NpletArgs a = base_args(c, r, (int)si);
      a.flag_ids = fids;
      a.flag_count = c->flag_counts + si;
      a.mode = 3;
      a.top_m = top_m;
      a.thr_keys = fz_keys(c) + (size_t)si * FUSE_NTHR;
      a.cand_ids = fz_ids(c);
      a.cand_b = fz_basis(c);
      a.cand_count = fz_counts(c) + (size_t)si * FUSE_NSEG;
      a.cand_cap = c->fz_cap;
      a.cand_nseg = FUSE_NSEG;
      a.cand_seg = c->fz_cap / FUSE_NSEG;
      a.cand_ws = fz_ws(c);
      a.part = c->part32 + p32_off;
      int grid = 0;
      st = prof_begin(c, s, 3);
      if (st != THOI_OK) return st;
      CK(launch_fused_sample(a, c->num_sms, s));
      st = prof_end(c, s);
      if (st != THOI_OK) return st;
      st = prof_begin(c, s, 0);
      if (st != THOI_OK) return st;
      CK(launch_nplet_f32(a, sh, c->num_sms, s, &grid, c->num_sms * MAX_BLOCKS_PER_SM_OUT));
      st = prof_end(c, s);
      if (st != THOI_OK) return st;
      p32_off += grid;
      md.g32 += grid;
      st = prof_begin(c, s, 3);
      if (st != THOI_OK) return st;
      CK(launch_reduce_candidates(a, c->num_sms, FUSE_CAND_BLOCKS, c->part32 + p32_off,
                                  top_m > 0 ? c->top32 + (size_t)p32_off * 2 * top_m : nullptr, s,
                                  &grid));
      st = prof_end(c, s);
      if (st != THOI_OK) return st;
      p32_off += grid;
      md.g32 += grid;
      md.thr_keys = a.thr_keys;
      md.status = c->status;
      launches += 2 + sel_kernels(top_m);  // sample, nplet kernel, candidate reduction
    } else if (red && !f64) {
      // FP32 records: basis values per piece, then the streaming reduction
      // each of the three arrays starts on a 256-byte boundary (16-byte loads)
      const unsigned long long bstride = basis_stride(maxn);
      for (unsigned long long a0 = r.r0; a0 < r.r1; a0 += PIECE) {
        SlotRange sub = r;
        sub.r0 = a0;
        sub.r1 = r.r1 - a0 > PIECE ? a0 + PIECE : r.r1;
        NpletArgs a = base_args(c, sub, (int)si);
        a.flag_ids = fids;
        a.flag_count = c->flag_counts + si;
        a.mode = 2;
        a.out = c->basis;
        a.out_f64 = 0;
        a.out_n = bstride;
        a.out_first = r.off + sub.r0;
        int grid = 0;
        st = prof_begin(c, s, 0);
        if (st != THOI_OK) return st;
        CK(launch_nplet_f32(a, sh, c->num_sms, s, &grid, c->num_sms * MAX_BLOCKS_PER_SM_OUT));
        st = prof_end(c, s);
        if (st != THOI_OK) return st;
        st = prof_begin(c, s, 3);
        if (st != THOI_OK) return st;
        const unsigned long long nsub = sub.r1 - sub.r0;
        if (sel && nsub <= FUSE_MIN_N) {
          CK(launch_select_basis(c->basis, bstride, nsub, r.off + sub.r0, md.cmb, top_m,
                                 c->sel_ws, c->status, c->part32 + p32_off,
                                 top_m > 0 ? c->top32 + (size_t)p32_off * 2 * top_m : nullptr,
                                 blk_cap, s, &grid));
          launches += 1 + sel_kernels(top_m);
        } else {
          CK(launch_reduce_basis(c->basis, bstride, nsub, r.off + sub.r0, md.cmb, top_m,
                                 c->seed_thr, c->part32 + p32_off,
                                 top_m > 0 ? c->top32 + (size_t)p32_off * 2 * top_m : nullptr,
                                 c->num_sms, blk_cap, s, &grid));
          // the nplet kernel, the reduction and (long ranges) its seed kernel
          launches += 2 + (top_m > 0 && nsub > (1ull << 20) && md.cmb.top != THOI_H ? 1 : 0);
        }
        st = prof_end(c, s);
        if (st != THOI_OK) return st;
        p32_off += grid;
        md.g32 += grid;
      }
    }
    if (red && f64 && f64s_threads(c->N, r.k, nullptr) > 0) {
      // FP64 records: basis values per piece, then the streaming reduction
      const unsigned long long bstride = basis_stride(maxn);
      for (unsigned long long a0 = r.r0; a0 < r.r1; a0 += PIECE) {
        SlotRange sub = r;
        sub.r0 = a0;
        sub.r1 = r.r1 - a0 > PIECE ? a0 + PIECE : r.r1;
        NpletArgs a = base_args(c, sub, (int)si);
        a.mode = 2;
        int grid = 0;
        st = prof_begin(c, s, 0);
        if (st != THOI_OK) return st;
        CK(launch_nplet_f64s(a, false, c->b64, bstride, c->num_sms, s, &grid,
                             c->num_sms * MAX_BLOCKS_PER_SM_OUT));
        st = prof_end(c, s);
        if (st != THOI_OK) return st;
        st = prof_begin(c, s, 3);
        if (st != THOI_OK) return st;
        if (sel64 && sub.r1 - sub.r0 <= FUSE_MIN_N) {
          // a short range by the radix select (ST_INEXACT: the caller repeats
          // the request without it)
          CK(launch_select_basis64(c->b64, bstride, sub.r1 - sub.r0, r.off + sub.r0, md.cmb,
                                   top_m, c->sel_ws, c->status, c->part32 + p32_off,
                                   top_m > 0 ? c->top32 + (size_t)p32_off * 2 * top_m : nullptr,
                                   blk_cap, s, &grid));
          launches += sel_kernels(top_m) - 1;
        } else {
          CK(launch_reduce_basis64(c->b64, bstride, sub.r1 - sub.r0, r.off + sub.r0, md.cmb,
                                   top_m, c->part32 + p32_off,
                                   top_m > 0 ? c->top32 + (size_t)p32_off * 2 * top_m : nullptr,
                                   c->num_sms, blk_cap, s, &grid));
        }
        st = prof_end(c, s);
        if (st != THOI_OK) return st;
        launches += 2;
        p32_off += grid;
        md.g32 += grid;
      }
    }
    const bool done_red = red && (!f64 || f64s_threads(c->N, r.k, nullptr) > 0);
    for (unsigned long long a0 = r.r0; a0 < r.r1 && !done_red; a0 += LAUNCH_SPLIT) {
      SlotRange sub = r;
      sub.r0 = a0;
      sub.r1 = r.r1 - a0 > LAUNCH_SPLIT ? a0 + LAUNCH_SPLIT : r.r1;
      NpletArgs a = base_args(c, sub, (int)si);
      a.flag_ids = fids;
      a.flag_count = c->flag_counts + si;
      a.mode = red ? 1 : 0;
      a.top_m = top_m;
      a.out = out_dev;
      a.out_f64 = c->opt.out_f64;
      a.out_n = id_end - id_begin;
      a.out_first = id_begin;
      a.part = red ? c->part32 + p32_off : nullptr;
      a.part_top = red && top_m > 0 ? c->top32 + (size_t)p32_off * 2 * top_m : nullptr;
      int grid = 0;
      const int cap = red ? blk_cap : c->num_sms * MAX_BLOCKS_PER_SM_OUT;
      st = prof_begin(c, s, 0);
      if (st != THOI_OK) return st;
      if (f64 && !red && f64s_threads(c->N, r.k, nullptr) > 0)
        CK(launch_nplet_f64s(a, false, nullptr, 0, c->num_sms, s, &grid, cap));
      else if (f64) CK(launch_nplet_f64(a, c->num_sms, s, &grid, cap));
      else CK(launch_nplet_f32(a, sh, c->num_sms, s, &grid, cap));
      st = prof_end(c, s);
      if (st != THOI_OK) return st;
      launches++;
      if (red) {
        p32_off += grid;
        md.g32 += grid;
      }
    }
    if (!f64 && r.r1 > r.r0) {
      // FP64 re-factor of this order's flagged nplets (count read on the device)
      cudaStream_t sr = s;
      if (overlap) {
        CK(cudaEventRecord(c->sev[2 * si], s));
        CK(cudaStreamWaitEvent(c->s2, c->sev[2 * si], 0));
        sr = c->s2;
      }
      NpletArgs a = base_args(c, r, (int)si);
      a.flag_ids = fids;
      a.flag_count = c->flag_counts + si;
      a.mode = red ? 1 : 0;
      a.top_m = top_m;
      a.out = out_dev;
      a.out_f64 = c->opt.out_f64;
      a.out_n = id_end - id_begin;
      a.out_first = id_begin;
      a.part = red ? c->part64 + p64_off : nullptr;
      a.part_top = red && top_m > 0 ? c->top64 + (size_t)p64_off * 2 * top_m : nullptr;
      int grid = 0;
      const bool smem_ok = f64s_threads(c->N, r.k, nullptr) > 0;
      if (smem_ok) {
        // FP64 kernel over the list, then (records) the list reduction
        const unsigned long long lstride = ((unsigned long long)c->flag_cap + 63) / 64 * 64;
        a.mode = red ? 2 : 0;
        st = prof_begin(c, sr, 1);
        if (st != THOI_OK) return st;
        CK(launch_nplet_f64s(a, true, fb64, lstride, c->num_sms, sr, &grid,
                             c->num_sms * MAX_BLOCKS_PER_SM_OUT));
        st = prof_end(c, sr);
        if (st != THOI_OK) return st;
        launches++;
        if (red) {
          st = prof_begin(c, sr, 3);
          if (st != THOI_OK) return st;
          if (sel) {
            CK(launch_select_list64(fb64, lstride, fids, c->flag_counts + si, c->flag_cap,
                                    md.cmb, top_m, c->sel_ws + sel_ws_bytes(), c->status,
                                    c->part64 + p64_off,
                                    top_m > 0 ? c->top64 + (size_t)p64_off * 2 * top_m : nullptr,
                                    ref_cap, sr, &grid));
            launches += sel_kernels(top_m) - 1;  // (one counted below)
          } else {
            // few blocks: the list is short next to the order, and each
            // block's top lists then cover enough entries for the merge to
            // keep few
            CK(launch_reduce_list64(fb64, lstride, fids, c->flag_counts + si, c->flag_cap,
                                    md.cmb, top_m, c->part64 + p64_off,
                                    top_m > 0 ? c->top64 + (size_t)p64_off * 2 * top_m : nullptr,
                                    c->num_sms, LIST_RED_BLOCKS, sr, &grid));
          }
          st = prof_end(c, sr);
          if (st != THOI_OK) return st;
          launches++;
        }
      } else {
        st = prof_begin(c, sr, 1);
        if (st != THOI_OK) return st;
        CK(launch_refactor(a, c->num_sms, sr, &grid, ref_cap));
        st = prof_end(c, sr);
        if (st != THOI_OK) return st;
        launches++;
      }
      if (overlap) CK(cudaEventRecord(c->sev[2 * si + 1], sr));
      if (red) {
        p64_off += grid;
        md.g64 = grid;
      }
    }
  }
  if (overlap) {
    // join: everything of the second stream before the merge and the return
    CK(cudaEventRecord(c->sev[2 * slots.size()], c->s2));
    CK(cudaStreamWaitEvent(s, c->sev[2 * slots.size()], 0));
  }
  if (red) {
    st = prof_begin(c, s, 2);
    if (st != THOI_OK) return st;
    CK(launch_merge(D, (int)slots.size(), c->part32, c->top32, c->part64, c->top64, top_m, recs_dev,
                    tops_dev, s));
    st = prof_end(c, s);
    if (st != THOI_OK) return st;
    launches++;
  }
  if (launches_out) *launches_out = launches;
  return THOI_OK;
}

extern "C" thoi_status thoi_measures(thoi_ctx* c, const int32_t* orders, int32_t n_orders,
                                     uint64_t id_begin, uint64_t id_end, int32_t kind, void* out,
                                     size_t out_bytes, thoi_stats* stats, void* stream) {
  if (!c || !orders_ok(c->N, orders, n_orders)) return THOI_ERR_INVALID_ARG;
  if (kind != THOI_RED_NONE && kind != THOI_RED_PER_ORDER) return THOI_ERR_INVALID_ARG;
  if (!out && !(kind == THOI_RED_NONE && id_begin == id_end)) return THOI_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<SlotRange> slots;
  uint64_t end = id_end;
  thoi_status st = plan_slots(c, orders, n_orders, id_begin, &end, &slots);
  if (st != THOI_OK) return st;
  const uint64_t n = end - id_begin;
  int launches = 0;
  if (kind == THOI_RED_NONE) {
    const size_t esz = c->opt.out_f64 ? 8 : 4;
    if (out_bytes < 5 * (size_t)n * esz) return THOI_ERR_INVALID_ARG;
    if (n > 0 && !is_device_ptr(out)) return THOI_ERR_INVALID_ARG;
    st = enqueue_measures(c, orders, n_orders, id_begin, end, kind, out, nullptr, nullptr, s,
                          &launches);
    if (st != THOI_OK) return st;
  } else {
    const size_t need = thoi_records_bytes(n_orders, c->opt.top_m);
    if (out_bytes < need) return THOI_ERR_INVALID_ARG;
    const bool dev = is_device_ptr(out);
    unsigned char* dst = (unsigned char*)out;
    if (!dev) {
      st = grow(&c->rec_buf, &c->rec_cap, need);
      if (st != THOI_OK) return st;
      dst = c->rec_buf;
    }
    thoi_order_record* recs = (thoi_order_record*)dst;
    TopEnt* tops = (TopEnt*)(dst + (size_t)n_orders * sizeof(thoi_order_record));
    // fused records first; a record the merge could not certify (or a full
    // candidate list) repeats the request with stored basis values
    for (int pass = 0; pass < 2; pass++) {
      st = enqueue_measures(c, orders, n_orders, id_begin, end, kind, nullptr, recs, tops, s,
                            &launches, pass == 0);
      if (st != THOI_OK) return st;
      if (!dev) CK(cudaMemcpyAsync(out, dst, need, cudaMemcpyDeviceToHost, s));
      int hs = 0;
      st = finish_status(c, s, (int)slots.size(), stats, n, launches, &hs);
      if (!(hs & (ST_INEXACT | ST_CAND_OVERFLOW)) || pass == 1) {
        if (stats && pass == 1) stats->fused_retries = 1;
        return st;
      }
    }
    return st;
  }
  return finish_status(c, s, (int)slots.size(), stats, n, launches);
}

// ------------------------------------------------------------------ API: gradient
extern "C" thoi_status thoi_measures_grad(thoi_ctx* c, const int32_t* orders, int32_t n_orders,
                                          int32_t measure, float* dL_dSigma, thoi_stats* stats,
                                          void* stream) {
  if (!c || !dL_dSigma || !orders_ok(c->N, orders, n_orders)) return THOI_ERR_INVALID_ARG;
  if (measure < THOI_H || measure > THOI_S) return THOI_ERR_INVALID_ARG;
  for (int i = 0; i < n_orders; i++)
    if (orders[i] > 32) return THOI_ERR_TOO_LARGE;
  if (!is_device_ptr(dL_dSigma)) return THOI_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<SlotRange> slots;
  uint64_t end = UINT64_MAX;
  thoi_status st = plan_slots(c, orders, n_orders, 0, &end, &slots);
  if (st != THOI_OK) return st;
  unsigned long long maxn = 0;
  for (auto& r : slots) maxn = (r.r1 - r.r0) > maxn ? (r.r1 - r.r0) : maxn;
  st = ensure_flag_ws(c, maxn);
  if (st != THOI_OK) return st;
  const int grid = c->num_sms * 4;
  const size_t NN = (size_t)c->N * c->N;
  st = grow(&c->gpart, &c->gpart_cap, (size_t)grid * NN);
  if (st != THOI_OK) return st;
  CK(cudaMemsetAsync(c->gpart, 0, (size_t)grid * NN * 8, s));
  CK(cudaMemsetAsync(c->status, 0, sizeof(int), s));
  CK(cudaMemsetAsync(c->flag_counts, 0, MAX_SLOTS * sizeof(unsigned long long), s));
  int launches = 0;
  for (size_t si = 0; si < slots.size(); si++) {
    const SlotRange& r = slots[si];
    if (r.r1 <= r.r0) continue;
    NpletArgs a = base_args(c, r);
    a.flag_count = c->flag_counts + si;
    const unsigned long long n = r.r1 - r.r0;
    int g = (int)((n + RED_NT - 1) / RED_NT);
    if (g > grid) g = grid;
    CK(launch_grad_pass(a, c->gpart, g, measure, false, s));
    CK(launch_grad_pass(a, c->gpart, c->num_sms, measure, true, s));
    launches += 2;
  }
  CK(launch_grad_finish(c->gpart, grid, c->sig64, c->N, dL_dSigma, s));
  launches++;
  return finish_status(c, s, (int)slots.size(), stats, thoi_count(c->N, orders, n_orders), launches);
}

// ------------------------------------------------------------------ API: group objectives
// Per order and piece of P_g ranks: every dataset's own path writes one
// measure per nplet (FP64) into row d of a D x P_g matrix (its FP64
// re-factor patching the row in place), a fold kernel keeps its status and
// re-factor count, then one kernel combines the D rows into the objective:
// the per-nplet output, or an FP64 basis piece fed to the FP64 streaming
// reduction; one merge at the end.
namespace {
// The D x P_g value matrix takes at most 16 GiB and a quarter of the free
// device memory: whole orders fit in one piece for the usual group sizes, so
// each dataset's pass can use the prefix-shared kernels.
constexpr unsigned long long GROUP_VALUE_BYTES = 1ull << 34;
constexpr unsigned long long GROUP_PIECE_MIN = 1ull << 16;
// streams for the datasets' passes: the passes of small orders are a few
// short launches each, which run side by side instead of one after another
constexpr int GROUP_STREAMS = 8;

// Options of the group's contexts, restored on every exit (a context may
// appear more than once: restored in reverse order).
struct GroupSaved {
  std::vector<std::pair<thoi_ctx*, thoi_options>> opt;
  std::vector<int> out_sel, top_meas;
  GroupSaved(thoi_ctx* const* ctxs, int D) {
    for (int d = 0; d < D; d++) {
      opt.push_back({ctxs[d], ctxs[d]->opt});
      out_sel.push_back(ctxs[d]->out_sel);
      top_meas.push_back(ctxs[d]->top_meas);
    }
  }
  ~GroupSaved() {
    for (int d = (int)opt.size() - 1; d >= 0; d--) {
      opt[d].first->opt = opt[d].second;
      opt[d].first->out_sel = out_sel[d];
      opt[d].first->top_meas = top_meas[d];
    }
  }
};

Combine group_combine() {
  Combine g;
  g.h_c = 0.0;
  g.tc_c = 0.0;
  g.dtc_c = 0.0;
  g.top = THOI_O;
  g.pad = 0;
  return g;
}
}  // namespace

static thoi_status group_args_ok(thoi_ctx* const* ctxs, int32_t D, int32_t measure,
                                 int32_t objective) {
  if (!ctxs || D < 1 || D > THOI_MAX_GROUP) return THOI_ERR_INVALID_ARG;
  for (int d = 0; d < D; d++)
    if (!ctxs[d] || ctxs[d]->N != ctxs[0]->N) return THOI_ERR_INVALID_ARG;
  if (measure < THOI_H || measure > THOI_S) return THOI_ERR_INVALID_ARG;
  if (objective == THOI_GROUP_MEAN) return THOI_OK;
  if (objective == THOI_GROUP_COHEN_D && D % 2 == 0 && D >= 4) return THOI_OK;
  return THOI_ERR_INVALID_ARG;
}

// Group status word and per-slot re-factor counters in ctxs[0]'s workspace.
static thoi_status group_meta(thoi_ctx* c0, cudaStream_t s, int** gstatus,
                              unsigned long long** gnref) {
  thoi_status st = grow(&c0->grp_meta, &c0->grp_meta_cap, (size_t)(1 + MAX_SLOTS) * 8);
  if (st != THOI_OK) return st;
  CK(cudaMemsetAsync(c0->grp_meta, 0, (size_t)(1 + MAX_SLOTS) * 8, s));
  *gstatus = (int*)c0->grp_meta;
  *gnref = (unsigned long long*)(c0->grp_meta + 8);
  return THOI_OK;
}

static thoi_status ensure_group_streams(thoi_ctx* c0, int ns) {
  while ((int)c0->gs.size() < ns) {
    cudaStream_t q;
    CK(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
    c0->gs.push_back(q);
  }
  while ((int)c0->gev.size() < ns + 1) {
    cudaEvent_t e;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    c0->gev.push_back(e);
  }
  return THOI_OK;
}

// Queue the group pass (no synchronisation); the caller has set the
// contexts' options (GroupSaved) and the group meta words.
static thoi_status enqueue_group(thoi_ctx* const* ctxs, int D, const int32_t* orders,
                                 int32_t n_orders, uint64_t id_begin, uint64_t id_end,
                                 int measure, int objective, int32_t kind, double* out_dev,
                                 thoi_order_record* recs_dev, TopEnt* tops_dev, int* gstatus,
                                 unsigned long long* gnref, cudaStream_t s, int* launches_out,
                                 uint64_t* evaluated) {
  thoi_ctx* c0 = ctxs[0];
  std::vector<SlotRange> slots;
  thoi_status st = plan_slots(c0, orders, n_orders, id_begin, &id_end, &slots);
  if (st != THOI_OK) return st;
  const bool red = kind == THOI_RED_PER_ORDER;
  const int top_m = red ? c0->opt.top_m : 0;
  unsigned long long maxn = 0;
  for (auto& r : slots) maxn = (r.r1 - r.r0) > maxn ? (r.r1 - r.r0) : maxn;
  size_t free_b = 0, total_b = 0;
  CK(cudaMemGetInfo(&free_b, &total_b));
  unsigned long long budget = GROUP_VALUE_BYTES;
  if ((unsigned long long)free_b / 4 < budget) budget = (unsigned long long)free_b / 4;
  unsigned long long piece = budget / (8ull * (unsigned long long)D);
  if (piece < GROUP_PIECE_MIN) piece = GROUP_PIECE_MIN;
  if (piece > maxn) piece = maxn > 0 ? maxn : 1;
  const unsigned long long ld = (piece + 63) / 64 * 64;
  st = grow(&c0->grp, &c0->grp_cap, (size_t)ld * (D + (red ? 3 : 0)));
  if (st != THOI_OK) return st;
  double* V = c0->grp;
  double* gb = c0->grp + (size_t)ld * D;
  const int blk_cap = c0->num_sms * MAX_BLOCKS_PER_SM_RED;
  if (red) {
    size_t n32 = 0;
    for (auto& r : slots) n32 += (size_t)((r.r1 - r.r0 + piece - 1) / piece) * blk_cap;
    st = ensure_parts(c0, n32, 1, top_m);
    if (st != THOI_OK) return st;
  }
  for (int d = 0; d < D; d++) {
    ctxs[d]->out_sel = measure + 1;
    ctxs[d]->opt.out_f64 = 1;
    ctxs[d]->opt.profile = 0;
  }
  // one stream per distinct context (a context listed twice keeps its
  // passes on one stream: they share its workspace), GROUP_STREAMS at most
  std::vector<int> sidx(D);
  int ns = 0;
  for (int d = 0; d < D; d++) {
    sidx[d] = -1;
    for (int e = 0; e < d; e++)
      if (ctxs[e] == ctxs[d]) sidx[d] = sidx[e];
    if (sidx[d] < 0) sidx[d] = ns++ % GROUP_STREAMS;
  }
  if (ns > GROUP_STREAMS) ns = GROUP_STREAMS;
  st = ensure_group_streams(c0, ns);
  if (st != THOI_OK) return st;
  const Combine cg = group_combine();
  MergeDescs MD;
  memset(&MD, 0, sizeof MD);
  int p32_off = 0, launches = 0;
  uint64_t ev = 0;
  for (size_t si = 0; si < slots.size(); si++) {
    const SlotRange& r = slots[si];
    MergeDesc& md = MD.d[si];
    md.k = r.k;
    md.cmb = cg;
    md.p32_off = p32_off;
    md.refactored = gnref + si;
    const int32_t k = r.k;
    for (unsigned long long a0 = r.r0; a0 < r.r1; a0 += piece) {
      const unsigned long long a1 = r.r1 - a0 > piece ? a0 + piece : r.r1;
      const unsigned long long n = a1 - a0;
      // fork: the datasets' passes on the group streams, joined before the
      // combine
      CK(cudaEventRecord(c0->gev[ns], s));
      for (int j = 0; j < ns; j++) CK(cudaStreamWaitEvent(c0->gs[j], c0->gev[ns], 0));
      for (int d = 0; d < D; d++) {
        thoi_ctx* cd = ctxs[d];
        cudaStream_t sd = c0->gs[sidx[d]];
        int nl = 0;
        st = enqueue_measures(cd, &k, 1, a0, a1, THOI_RED_NONE, V + (size_t)d * ld, nullptr,
                              nullptr, sd, &nl);
        if (st != THOI_OK) return st;
        CK(launch_group_fold(cd->status, cd->flag_counts, cd->flag_cap, gstatus, gnref + si, sd));
        launches += nl + 1;
      }
      for (int j = 0; j < ns; j++) {
        CK(cudaEventRecord(c0->gev[j], c0->gs[j]));
        CK(cudaStreamWaitEvent(s, c0->gev[j], 0));
      }
      ev += n * (uint64_t)D;
      CK(launch_group_combine(V, ld, n, nullptr, D, objective,
                              red ? nullptr : out_dev + (r.off + a0 - id_begin),
                              red ? gb : nullptr, ld, c0->num_sms, s));
      launches++;
      if (red) {
        int grid = 0;
        CK(launch_reduce_basis64(gb, ld, n, r.off + a0, cg, top_m, c0->part32 + p32_off,
                                 top_m > 0 ? c0->top32 + (size_t)p32_off * 2 * top_m : nullptr,
                                 c0->num_sms, blk_cap, s, &grid));
        launches++;
        p32_off += grid;
        md.g32 += grid;
      }
    }
  }
  if (red) {
    CK(launch_merge(MD, (int)slots.size(), c0->part32, c0->top32, c0->part64, c0->top64, top_m,
                    recs_dev, tops_dev, s));
    CK(launch_group_fix(recs_dev, (int)slots.size(), s));
    launches += 2;
  }
  if (launches_out) *launches_out = launches;
  if (evaluated) *evaluated = ev;
  return THOI_OK;
}

static thoi_status group_finish(thoi_ctx* c0, cudaStream_t s, const int* gstatus,
                                const unsigned long long* gnref, int n_slots, thoi_stats* stats,
                                uint64_t evaluated, int launches) {
  int hs = 0;
  unsigned long long nr[MAX_SLOTS];
  CK(cudaMemcpyAsync(&hs, gstatus, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (n_slots > 0)
    CK(cudaMemcpyAsync(nr, gnref, (size_t)n_slots * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (stats) {
    memset(stats, 0, sizeof *stats);
    stats->nplets = evaluated;
    for (int i = 0; i < n_slots; i++) stats->n_refactored += nr[i];
    stats->launches = launches;
  }
  (void)c0;
  if (hs & ST_FLAG_OVERFLOW) return THOI_ERR_WORKSPACE;
  if (hs & ST_CANCELLED) return THOI_ERR_CANCELLED;
  if (hs & ST_NOT_PD) return THOI_ERR_NOT_PD;
  return THOI_OK;
}

extern "C" thoi_status thoi_group_measures(thoi_ctx* const* ctxs, int32_t D, const int32_t* orders,
                                           int32_t n_orders, uint64_t id_begin, uint64_t id_end,
                                           int32_t measure, int32_t objective, int32_t kind,
                                           void* out, size_t out_bytes, thoi_stats* stats,
                                           void* stream) {
  thoi_status st = group_args_ok(ctxs, D, measure, objective);
  if (st != THOI_OK) return st;
  thoi_ctx* c0 = ctxs[0];
  if (!orders_ok(c0->N, orders, n_orders)) return THOI_ERR_INVALID_ARG;
  if (kind != THOI_RED_NONE && kind != THOI_RED_PER_ORDER) return THOI_ERR_INVALID_ARG;
  if (!out && !(kind == THOI_RED_NONE && id_begin == id_end)) return THOI_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<SlotRange> slots;
  uint64_t end = id_end;
  st = plan_slots(c0, orders, n_orders, id_begin, &end, &slots);
  if (st != THOI_OK) return st;
  const uint64_t n = end - id_begin;
  int* gstatus = nullptr;
  unsigned long long* gnref = nullptr;
  st = group_meta(c0, s, &gstatus, &gnref);
  if (st != THOI_OK) return st;
  GroupSaved saved(ctxs, D);
  int launches = 0;
  uint64_t ev = 0;
  if (kind == THOI_RED_NONE) {
    if (out_bytes < (size_t)n * 8) return THOI_ERR_INVALID_ARG;
    if (n > 0 && !is_device_ptr(out)) return THOI_ERR_INVALID_ARG;
    st = enqueue_group(ctxs, D, orders, n_orders, id_begin, end, measure, objective, kind,
                       (double*)out, nullptr, nullptr, gstatus, gnref, s, &launches, &ev);
    if (st != THOI_OK) return st;
  } else {
    const size_t need = thoi_records_bytes(n_orders, c0->opt.top_m);
    if (out_bytes < need) return THOI_ERR_INVALID_ARG;
    const bool dev = is_device_ptr(out);
    unsigned char* dst = (unsigned char*)out;
    if (!dev) {
      st = grow(&c0->rec_buf, &c0->rec_cap, need);
      if (st != THOI_OK) return st;
      dst = c0->rec_buf;
    }
    thoi_order_record* recs = (thoi_order_record*)dst;
    TopEnt* tops = (TopEnt*)(dst + (size_t)n_orders * sizeof(thoi_order_record));
    st = enqueue_group(ctxs, D, orders, n_orders, id_begin, end, measure, objective, kind,
                       nullptr, recs, tops, gstatus, gnref, s, &launches, &ev);
    if (st != THOI_OK) return st;
    if (!dev) CK(cudaMemcpyAsync(out, dst, need, cudaMemcpyDeviceToHost, s));
  }
  return group_finish(c0, s, gstatus, gnref, (int)slots.size(), stats, ev, launches);
}

// ------------------------------------------------------------------ API: batch
// Multi-dataset batch plan: descriptors, workspace and the CUDA graph of one
// (contexts, kmin, kmax) combination.  Every (dataset d, order k <= N_d)
// pair is a slot; every slot is cut into tiles of BATCH_TILE ranks.  The
// tiles of all slots form one list, largest orders first, and one launch of
// the persistent batched kernel per band of orders (one launch when kmax <=
// 8) evaluates and reduces them all, each tile into its own partial record.
// Then, per order, the batched FP64 re-factor of the flagged nplets; one list
// reduction over every slot; one merge over every (dataset, order) pair.
// Plans are cached by context serial numbers, so a repeated call replays the
// graph.
namespace {

constexpr unsigned long long BATCH_TILE = 1ull << 16;
constexpr int BATCH_CACHE = 4;

struct BatchPlan {
  std::vector<unsigned long long> serials;
  int kmin = 0, kmax = 0, top_m = 0, device = 0;
  unsigned long long tune_gen = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<void*> allocs;
  unsigned char* staging = nullptr;
  size_t per = 0;
  int* status = nullptr;
  unsigned long long* flag_counts = nullptr;
  std::vector<unsigned long long> flag_caps;
  int n_slots = 0;
  int launches = 0;
  int nplet_launches = 0;
  unsigned long long nplets = 0;
};

void plan_free(BatchPlan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  for (void* q : p->allocs) cudaFree(q);
  delete p;
}

}  // namespace

static std::mutex g_batch_mu;
static std::vector<BatchPlan*> g_batch;  // most recently used last
static unsigned long long g_serial = 0;  // guarded by g_batch_mu

static unsigned long long next_serial() {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  return ++g_serial;
}

static void batch_forget(unsigned long long serial) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (size_t i = 0; i < g_batch.size();) {
    bool hit = false;
    for (auto x : g_batch[i]->serials) hit |= x == serial;
    if (hit) {
      plan_free(g_batch[i]);
      g_batch.erase(g_batch.begin() + i);
    } else {
      i++;
    }
  }
}

template <typename T>
static thoi_status plan_alloc(BatchPlan* p, T** ptr, size_t n) {
  void* q = nullptr;
  CK(cudaMalloc(&q, (n > 0 ? n : 1) * sizeof(T)));
  p->allocs.push_back(q);
  *ptr = (T*)q;
  return THOI_OK;
}

static int batch_band_of(int k) {
  for (int b = 0; b < BATCH_BANDS; b++)
    if (k >= BATCH_BAND_LO[b] && k <= BATCH_BAND_HI[b]) return b;
  return -1;
}

// Autotune cache key of the batched kernel's per-order chunk (nplets per
// thread per round), tuned on a batch: GPU, SM count, order, mask width.
static std::string batch_tune_key(const char* gpu, int sms, int k, int wide) {
  return tune_key(gpu, sms, k, wide) + "|batch";
}

// Time the batched kernel on the tiles [t0, t1) of one order with each
// chunk in {1, 2, 4, 8} (after a warm-up run) and cache the fastest.
static thoi_status batch_tune_order(thoi_ctx* c0, int k, bool wide, BatchFArgs b,
                                    const BatchFTile* d_tiles, int t0, int t1, int maxN,
                                    unsigned* counter) {
  cudaStream_t s = nullptr;
  CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  int best_chunk = 8;
  float best = -1.f;
  const int chunks[4] = {8, 4, 2, 1};
  b.tiles = d_tiles + t0;
  b.n_tiles = t1 - t0;
  b.tile_counter = counter;
  for (int ci = 0; ci < 4 && e == cudaSuccess; ci++) {
    b.chunk_k[k] = chunks[ci];
    for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {
      e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
      if (e == cudaSuccess) e = cudaEventRecord(e0, s);
      if (e == cudaSuccess)
        e = launch_batch_fused(batch_band_of(k), wide, b, maxN, 0, c0->num_sms, s, nullptr);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float t = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
      if (e == cudaSuccess && rep == 1 && (best < 0.f || t < best)) {
        best = t;
        best_chunk = chunks[ci];
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  if (e != cudaSuccess) return cuda_fail(e);
  Shape sh;
  sh.blocks_per_sm = 0;
  sh.chunk = best_chunk;
  sh.lanes = 1;
  sh.prefix = 0;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_batch[batch_tune_key(c0->gpu_name, c0->num_sms, k, wide)] = sh;
  return THOI_OK;
}

static thoi_status batch_build(thoi_ctx* const* ctxs, int D, int kmin, int kmax,
                               BatchPlan* P) {
  cudaStream_t s = nullptr;
  thoi_ctx* c0 = ctxs[0];
  const int top_m = c0->opt.top_m;
  const int no = kmax - kmin + 1;
  const int num_sms = c0->num_sms;
  int maxN = 0;
  for (int d = 0; d < D; d++) maxN = ctxs[d]->N > maxN ? ctxs[d]->N : maxN;
  const bool wide = maxN > 32;
  // datasets
  std::vector<BatchDataset> hds(D);
  for (int d = 0; d < D; d++) {
    const thoi_ctx* c = ctxs[d];
    hds[d].R32 = c->R32;
    hds[d].R64 = c->R64;
    hds[d].ls = c->ls;
    hds[d].N = c->N;
    hds[d].tau_piv = c->opt.pivot_tau;
    hds[d].tau_tr = c->opt.trace_tau;
    hds[d].pad = 0;
  }
  // slots by order; every slot has its own region of the flag list (all
  // orders run in one launch)
  std::vector<BatchSlot> hsl;
  std::vector<int> slot0(no, 0), nslot(no, 0);
  std::vector<int> slot_of(D * no, -1);  // (d, q) -> slot
  unsigned long long foff = 0;
  for (int q = 0; q < no; q++) {
    const int k = kmin + q;
    slot0[q] = (int)hsl.size();
    for (int d = 0; d < D; d++) {
      const thoi_ctx* c = ctxs[d];
      if (k > c->N) continue;
      BatchSlot sl;
      memset(&sl, 0, sizeof sl);
      sl.d = d;
      sl.k = k;
      sl.n = binom_host(c->N, k);
      unsigned long long ib = 0;
      for (int kk = kmin; kk < k; kk++) ib += binom_host(c->N, kk);
      sl.id_base = ib;
      unsigned long long cap;
      if (c->opt.flag_capacity > 0) {
        cap = c->opt.flag_capacity;
      } else {
        cap = sl.n / 16 + 1;
        if (cap < (1ull << 16)) cap = 1ull << 16;
      }
      if (cap > sl.n) cap = sl.n;
      sl.flag_off = foff;
      sl.flag_cap = cap;
      foff += (cap + 63) / 64 * 64;
      sl.cmb = combine_for(c, k);
      slot_of[d * no + q] = (int)hsl.size();
      hsl.push_back(sl);
      P->nplets += sl.n;
    }
    nslot[q] = (int)hsl.size() - slot0[q];
  }
  const unsigned long long lstride = foff > 64 ? foff : 64;
  const int n_slots = (int)hsl.size();
  P->n_slots = n_slots;
  for (auto& sl : hsl) P->flag_caps.push_back(sl.flag_cap);
  // tiles: partial indices slot-major (a slot's partials are contiguous),
  // list order by order descending (then slot)
  std::vector<BatchFTile> htiles;
  std::vector<int> pfirst(n_slots, 0), pcount(n_slots, 0);
  int np = 0;
  for (int si = 0; si < n_slots; si++) {
    pfirst[si] = np;
    for (unsigned long long r0 = 0; r0 < hsl[si].n; r0 += BATCH_TILE) {
      BatchFTile t;
      t.r0 = r0;
      t.n = (unsigned)(hsl[si].n - r0 < BATCH_TILE ? hsl[si].n - r0 : BATCH_TILE);
      t.slot = si;
      t.pidx = np++;
      t.k = hsl[si].k;
      htiles.push_back(t);
    }
    pcount[si] = np - pfirst[si];
  }
  std::stable_sort(htiles.begin(), htiles.end(),
                   [](const BatchFTile& a, const BatchFTile& b) { return a.k > b.k; });
  // band ranges of the sorted list
  int band_t0[BATCH_BANDS], band_t1[BATCH_BANDS];
  for (int b = 0; b < BATCH_BANDS; b++) band_t0[b] = band_t1[b] = 0;
  for (int b = 0; b < BATCH_BANDS; b++) {
    int t0 = -1, t1 = -1;
    for (int t = 0; t < (int)htiles.size(); t++)
      if (batch_band_of(htiles[t].k) == b) {
        if (t0 < 0) t0 = t;
        t1 = t + 1;
      }
    if (t0 >= 0) {
      band_t0[b] = t0;
      band_t1[b] = t1;
    }
  }
  // merge descriptors: every (dataset, order) pair, records in output order;
  // FP64 list partials: B2 blocks per slot
  const int B2 = [&]() {
    int b = n_slots > 0 ? (2 * num_sms) / n_slots : 1;
    if (b < 1) b = 1;
    if (b > 8) b = 8;
    return b;
  }();
  const size_t per = thoi_records_bytes(no, top_m);
  P->per = per;
  std::vector<MergeDesc> hmd(D * no);
  int gmax = 1;
  for (int d = 0; d < D; d++) {
    for (int q = 0; q < no; q++) {
      MergeDesc& m = hmd[d * no + q];
      memset(&m, 0, sizeof m);
      m.k = kmin + q;
      const int si = slot_of[d * no + q];
      if (si >= 0) {
        m.p32_off = pfirst[si];
        m.g32 = pcount[si];
        m.p64_off = si * B2;
        m.g64 = B2;
        m.cmb = hsl[si].cmb;
      }
      if (m.g32 + m.g64 > gmax) gmax = m.g32 + m.g64;
    }
  }
  // device buffers
  thoi_status st;
  BatchDataset* d_ds;
  BatchSlot* d_sl;
  BatchFTile* d_tiles;
  MergeDesc* d_md;
  thoi_order_record** d_recp;
  TopEnt** d_topp;
  double* b64;
  unsigned long long* flag_ids;
  PartRec *part32, *part64;
  TopEnt *top32, *top64;
  unsigned* counters;
  unsigned* slot_thr;
  const size_t n64 = (size_t)n_slots * B2;
  if ((st = plan_alloc(P, &d_ds, D)) != THOI_OK) return st;
  if ((st = plan_alloc(P, &d_sl, n_slots)) != THOI_OK) return st;
  if ((st = plan_alloc(P, &d_tiles, htiles.size())) != THOI_OK) return st;
  if ((st = plan_alloc(P, &d_md, hmd.size())) != THOI_OK) return st;
  if ((st = plan_alloc(P, &d_recp, hmd.size())) != THOI_OK) return st;
  if ((st = plan_alloc(P, &d_topp, hmd.size())) != THOI_OK) return st;
  if ((st = plan_alloc(P, &b64, 3 * (size_t)lstride)) != THOI_OK) return st;
  if ((st = plan_alloc(P, &flag_ids, (size_t)lstride)) != THOI_OK) return st;
  if ((st = plan_alloc(P, &P->flag_counts, (size_t)n_slots)) != THOI_OK) return st;
  if ((st = plan_alloc(P, &part32, (size_t)np)) != THOI_OK) return st;
  if ((st = plan_alloc(P, &part64, n64)) != THOI_OK) return st;
  if ((st = plan_alloc(P, &top32, (size_t)np * 2 * (size_t)top_m)) != THOI_OK) return st;
  if ((st = plan_alloc(P, &top64, n64 * 2 * (size_t)top_m)) != THOI_OK) return st;
  if ((st = plan_alloc(P, &P->staging, per * (size_t)D)) != THOI_OK) return st;
  if ((st = plan_alloc(P, &P->status, 1)) != THOI_OK) return st;
  if ((st = plan_alloc(P, &counters, BATCH_BANDS + 1)) != THOI_OK) return st;
  if ((st = plan_alloc(P, &slot_thr, 2 * (size_t)(n_slots > 0 ? n_slots : 1))) != THOI_OK)
    return st;
  for (int d = 0; d < D; d++) {
    for (int q = 0; q < no; q++) {
      const int si = slot_of[d * no + q];
      if (si >= 0) hmd[d * no + q].refactored = P->flag_counts + si;
    }
  }
  std::vector<thoi_order_record*> hrecp(hmd.size());
  std::vector<TopEnt*> htopp(hmd.size());
  for (int d = 0; d < D; d++)
    for (int q = 0; q < no; q++) {
      unsigned char* base = P->staging + per * d;
      hrecp[d * no + q] = (thoi_order_record*)base + q;
      htopp[d * no + q] =
          (TopEnt*)(base + (size_t)no * sizeof(thoi_order_record)) + (size_t)q * 2 * top_m;
    }
  CK(cudaMemcpy(d_ds, hds.data(), hds.size() * sizeof(BatchDataset), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_sl, hsl.data(), hsl.size() * sizeof(BatchSlot), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_tiles, htiles.data(), htiles.size() * sizeof(BatchFTile),
                cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_md, hmd.data(), hmd.size() * sizeof(MergeDesc), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_recp, hrecp.data(), hrecp.size() * sizeof(void*), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_topp, htopp.data(), htopp.size() * sizeof(void*), cudaMemcpyHostToDevice));
  // kernel arguments; per-order chunks from the batch autotune cache, tuned
  // here on this batch where missing (when the contexts autotune)
  BatchFArgs ba;
  memset(&ba, 0, sizeof ba);
  ba.ds = d_ds;
  ba.slots = d_sl;
  ba.top_m = top_m;
  ba.binom = c0->binom;
  ba.flag_ids = flag_ids;
  ba.flag_counts = P->flag_counts;
  ba.part = part32;
  ba.part_top = top32;
  ba.status = P->status;
  ba.cancel = c0->d_cancel;
  for (int k = 0; k <= KBATCH_MAX; k++) ba.chunk_k[k] = 8;
  for (int q = 0; q < no; q++) {
    const int k = kmin + q;
    if (nslot[q] == 0) continue;
    bool have = false;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune_batch.find(batch_tune_key(c0->gpu_name, num_sms, k, wide));
      if (it != g_tune_batch.end()) {
        ba.chunk_k[k] = it->second.chunk;
        have = true;
      }
    }
    if (!have && c0->opt.autotune) {
      int t0 = -1, t1 = -1;
      for (int t = 0; t < (int)htiles.size(); t++)
        if (htiles[t].k == k) {
          if (t0 < 0) t0 = t;
          t1 = t + 1;
        }
      if (t0 >= 0) {
        st = batch_tune_order(c0, k, wide, ba, d_tiles, t0, t1, maxN, counters + BATCH_BANDS);
        if (st != THOI_OK) return st;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        ba.chunk_k[k] = g_tune_batch[batch_tune_key(c0->gpu_name, num_sms, k, wide)].chunk;
      }
    }
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    P->tune_gen = g_tune_gen;
  }
  // capture on a private stream (the caller's may be the legacy default
  // stream, which cannot be captured); the graph is launched on the caller's
  int nl = 0, nnl = 0;
  cudaStream_t cs = nullptr;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  s = cs;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaStreamDestroy(cs);
    return cuda_fail(cudaGetLastError());
  }
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) {
    if (e == cudaSuccess && x != cudaSuccess) e = x;
    return e == cudaSuccess;
  };
  ok(cudaMemsetAsync(P->status, 0, sizeof(int), s));
  ok(cudaMemsetAsync(P->flag_counts, 0, (size_t)(n_slots > 0 ? n_slots : 1) * 8, s));
  ok(cudaMemsetAsync(counters, 0, (BATCH_BANDS + 1) * sizeof(unsigned), s));
  ok(cudaMemsetAsync(slot_thr, 0, 2 * (size_t)(n_slots > 0 ? n_slots : 1) * sizeof(unsigned), s));
  // the nplets: one persistent launch per band, largest orders first
  for (int b = BATCH_BANDS - 1; b >= 0 && e == cudaSuccess; b--) {
    if (band_t1[b] <= band_t0[b]) continue;
    BatchFArgs bb = ba;
    bb.tiles = d_tiles + band_t0[b];
    bb.n_tiles = band_t1[b] - band_t0[b];
    bb.tile_counter = counters + b;
    bb.slot_thr = slot_thr;
    ok(launch_batch_fused(b, wide, bb, maxN, 0, num_sms, s, nullptr));
    nl++;
    nnl++;
  }
  // FP64 re-factor of the flagged nplets, per order (its launch shape depends
  // on k), then one list reduction over every slot
  for (int q = 0; q < no && e == cudaSuccess; q++) {
    if (nslot[q] == 0) continue;
    const int k = kmin + q;
    int bx = (2 * num_sms) / nslot[q];
    if (bx < 1) bx = 1;
    if (bx > 64) bx = 64;
    ok(launch_refactor_batch(d_ds, d_sl, slot0[q], nslot[q], maxN, k, wide, c0->binom, flag_ids,
                             P->flag_counts, b64, lstride, P->status, bx, s));
    nl++;
  }
  ok(launch_reduce_list_batch(b64, lstride, d_sl, 0, n_slots, flag_ids, P->flag_counts, top_m,
                              part64, top64, B2, s));
  nl++;
  ok(launch_merge_arr(d_md, D * no, gmax, part32, top32, part64, top64, top_m, d_recp, d_topp, s));
  nl++;
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(s, &g);
  cudaStreamDestroy(cs);
  if (e == cudaSuccess) e = ee;
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return cuda_fail(e);
  }
  P->graph = g;
  CK(cudaGraphInstantiate(&P->exec, g, 0));
  P->launches = nl;
  P->nplet_launches = nnl;
  return THOI_OK;
}

static thoi_status batch_graph(thoi_ctx* const* ctxs, int32_t D, int32_t kmin, int32_t kmax,
                               void* out, thoi_stats* stats, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  thoi_ctx* c0 = ctxs[0];
  std::vector<unsigned long long> key(D);
  for (int d = 0; d < D; d++) key[d] = ctxs[d]->serial;
  BatchPlan* P = nullptr;
  unsigned long long tg;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tg = g_tune_gen;
  }
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (size_t i = 0; i < g_batch.size(); i++) {
    BatchPlan* p = g_batch[i];
    if (p->serials == key && p->kmin == kmin && p->kmax == kmax && p->device == c0->device &&
        p->tune_gen == tg) {
      P = p;
      g_batch.erase(g_batch.begin() + i);
      g_batch.push_back(P);
      break;
    }
  }
  if (!P) {
    P = new BatchPlan;
    P->serials = key;
    P->kmin = kmin;
    P->kmax = kmax;
    P->top_m = c0->opt.top_m;
    P->device = c0->device;
    const thoi_status st = batch_build(ctxs, D, kmin, kmax, P);
    if (st != THOI_OK) {
      plan_free(P);
      return st;
    }
    while ((int)g_batch.size() >= BATCH_CACHE) {
      plan_free(g_batch.front());
      g_batch.erase(g_batch.begin());
    }
    g_batch.push_back(P);
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c0->opt.profile) {
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, s));
  }
  CK(cudaGraphLaunch(P->exec, s));
  if (e1) CK(cudaEventRecord(e1, s));
  CK(cudaMemcpyAsync(out, P->staging, P->per * (size_t)D, cudaMemcpyDefault, s));
  int hs = 0;
  std::vector<unsigned long long> fc(P->n_slots > 0 ? P->n_slots : 1);
  CK(cudaMemcpyAsync(&hs, P->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(fc.data(), P->flag_counts, fc.size() * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  float ms = 0.f;
  if (e1) {
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  if (stats) {
    memset(stats, 0, sizeof *stats);
    unsigned long long nref = 0;
    for (int i = 0; i < P->n_slots; i++) nref += fc[i] < P->flag_caps[i] ? fc[i] : P->flag_caps[i];
    stats->nplets = P->nplets;
    stats->n_refactored = nref;
    stats->launches = P->launches;
    stats->nplet_launches = P->nplet_launches;
    stats->nplet_ms = ms;
  }
  if (hs & ST_FLAG_OVERFLOW) return THOI_ERR_WORKSPACE;
  if (hs & ST_CANCELLED) return THOI_ERR_CANCELLED;
  if (hs & ST_NOT_PD) return THOI_ERR_NOT_PD;
  return THOI_OK;
}

// One context after the other through thoi_measures (FP64 path, or orders
// above the register kernels' range).
static thoi_status batch_sequential(thoi_ctx* const* ctxs, int32_t D, int32_t kmin, int32_t kmax,
                                    void* out, thoi_stats* stats, void* stream) {
  const int top_m = ctxs[0]->opt.top_m;
  const int no = kmax - kmin + 1;
  const size_t per = thoi_records_bytes(no, top_m);
  const bool dev = is_device_ptr(out);
  std::vector<unsigned char> host(per);
  thoi_stats tot;
  memset(&tot, 0, sizeof tot);
  for (int d = 0; d < D; d++) {
    thoi_ctx* c = ctxs[d];
    std::vector<int32_t> ords;
    for (int k = kmin; k <= kmax && k <= c->N; k++) ords.push_back(k);
    memset(host.data(), 0, per);
    thoi_order_record* R = (thoi_order_record*)host.data();
    thoi_top_entry* Tp = (thoi_top_entry*)(host.data() + (size_t)no * sizeof(thoi_order_record));
    for (int q = 0; q < no; q++) {
      R[q].k = kmin + q;
      for (int m = 0; m < 5; m++) R[q].argmin[m] = R[q].argmax[m] = ~0ull;
    }
    for (size_t q = 0; q < (size_t)no * 2 * top_m; q++) Tp[q].id = ~0ull;
    if (!ords.empty()) {
      const int nv = (int)ords.size();
      std::vector<unsigned char> tmp(thoi_records_bytes(nv, top_m));
      thoi_stats st1;
      thoi_status st = thoi_measures(c, ords.data(), nv, 0, UINT64_MAX, THOI_RED_PER_ORDER,
                                     tmp.data(), tmp.size(), &st1, stream);
      if (st != THOI_OK) return st;
      memcpy(R, tmp.data(), (size_t)nv * sizeof(thoi_order_record));
      const thoi_top_entry* tt = (const thoi_top_entry*)(tmp.data() + (size_t)nv * sizeof(thoi_order_record));
      memcpy(Tp, tt, (size_t)nv * 2 * top_m * sizeof(thoi_top_entry));
      tot.nplets += st1.nplets;
      tot.n_refactored += st1.n_refactored;
      tot.launches += st1.launches;
    }
    unsigned char* dst = (unsigned char*)out + per * d;
    if (dev) CK(cudaMemcpy(dst, host.data(), per, cudaMemcpyHostToDevice));
    else memcpy(dst, host.data(), per);
  }
  if (stats) *stats = tot;
  return THOI_OK;
}


extern "C" thoi_status thoi_batch_measures(thoi_ctx* const* ctxs, int32_t D, int32_t kmin,
                                           int32_t kmax, void* out, size_t out_bytes,
                                           thoi_stats* stats, void* stream) {
  if (!ctxs || D < 1 || kmin < 1 || kmax < kmin || kmax > THOI_MAX_N || !out)
    return THOI_ERR_INVALID_ARG;
  const int top_m = ctxs[0]->opt.top_m;
  const int prec = ctxs[0]->opt.precision;
  for (int d = 0; d < D; d++)
    if (!ctxs[d] || ctxs[d]->opt.top_m != top_m || ctxs[d]->opt.precision != prec ||
        ctxs[d]->device != ctxs[0]->device)
      return THOI_ERR_INVALID_ARG;
  const int no = kmax - kmin + 1;
  if (out_bytes < thoi_records_bytes(no, top_m) * (size_t)D) return THOI_ERR_INVALID_ARG;
  // the batched kernels cover the FP32 path up to the register kernels' order
  int top_k = 0;
  for (int d = 0; d < D; d++) {
    const int kk = kmax < ctxs[d]->N ? kmax : ctxs[d]->N;
    top_k = kk > top_k ? kk : top_k;
  }
  if (prec != THOI_F32_FIX64 || top_k > KBATCH_MAX || D > 65535)
    return batch_sequential(ctxs, D, kmin, kmax, out, stats, stream);
  return batch_graph(ctxs, D, kmin, kmax, out, stats, stream);
}

// ------------------------------------------------------------------ API: greedy search
// Greedy search (Methods, "Heuristics", "Greedy Algorithm"): the kappa best
// nplets of order k0 by an exhaustive pass, then order by order every
// selected set grows by each variable it lacks, the distinct candidates are
// evaluated, and the kappa best become the next selection.  Evaluation in the
// FP64 path on the device (shared-memory FP64 kernels), selection on the
// device by the per-block top lists and their merge, ranked by one measure;
// ties go to the smallest lexicographic rank.  The candidate sets (at most
// kappa * N per order) are formed and de-duplicated on the device too.
static uint64_t rank_to_mask(int N, int k, uint64_t rank) {
  int32_t idx[THOI_MAX_N];
  int32_t kk = 0;
  const int32_t ord = k;
  if (thoi_unrank(N, &ord, 1, rank, idx, &kk) != THOI_OK) return 0;
  uint64_t m = 0;
  for (int i = 0; i < kk; i++) m |= 1ull << idx[i];
  return m;
}

// Greedy search on one context's measure (objective < 0) or on a group
// objective over D contexts.  Every order runs on the stream: the exhaustive
// records of order k0, then per order the device expansion of the selected
// sets (k_greedy_expand), the FP64 list evaluation, the list reduction and
// the merge into that order's records; the host reads all orders' top lists
// once at the end.
// sel: each order's list reduced by the radix select (else by the streaming
// reduction, which the search falls back to when a select gathers too many
// tied entries).
static thoi_status greedy_impl(thoi_ctx* const* ctxs, int D, int objective, int32_t k0,
                               int32_t k1, int32_t kappa, int32_t measure, int32_t maximize,
                               uint64_t* sets_out, double* values_out, thoi_stats* stats,
                               cudaStream_t s, bool sel = true) {
  thoi_ctx* c = ctxs[0];
  const bool group = objective >= 0;
  const int N = c->N;
  const int side = maximize ? 0 : 1;
  const int levels = k1 - k0 + 1;
  for (size_t q = 0; q < (size_t)levels * kappa; q++) {
    sets_out[q] = 0;
    values_out[q] = NAN;
  }
  // every context runs the FP64 path; the first ranks its top lists (kappa
  // entries) by the measure, or holds the group's; restored on every exit
  GroupSaved saved(ctxs, D);
  for (int d = 0; d < D; d++) {
    ctxs[d]->opt.precision = THOI_F64;
    ctxs[d]->opt.profile = 0;
  }
  c->opt.top_m = kappa;
  c->top_meas = measure;
  int* gstatus = nullptr;
  unsigned long long* gnref = nullptr;
  thoi_status st = THOI_OK;
  if (group) {
    st = group_meta(c, s, &gstatus, &gnref);
    if (st != THOI_OK) return st;
  }
  // device buffers of the whole search
  const int ref_cap = c->num_sms * REFACTOR_BLOCKS_PER_SM;
  const size_t cap = (size_t)kappa * N;
  const size_t lstride = (cap + 63) / 64 * 64;
  size_t tsize = 1;
  while (tsize < 2 * cap) tsize <<= 1;
  const size_t per_level = sizeof(thoi_order_record) + 2 * (size_t)kappa * sizeof(TopEnt);
  struct Bufs {
    void* p[7];
    ~Bufs() {
      for (void* q : p) if (q) cudaFree(q);
    }
  } bufs{{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr}};
  PartRec* part = nullptr;
  TopEnt* ptop = nullptr;
  unsigned long long* d_ids = nullptr;
  unsigned long long* d_cnt = nullptr;  // candidates per order
  double* b64 = nullptr;
  unsigned long long* table = nullptr;
  unsigned char* d_lv = nullptr;        // per order: record, then 2 x kappa top entries
  CK(cudaMalloc(&part, ref_cap * sizeof(PartRec)));
  bufs.p[0] = part;
  CK(cudaMalloc(&ptop, (size_t)ref_cap * 2 * kappa * sizeof(TopEnt)));
  bufs.p[1] = ptop;
  CK(cudaMalloc(&d_ids, cap * sizeof(unsigned long long)));
  bufs.p[2] = d_ids;
  CK(cudaMalloc(&d_cnt, (size_t)levels * sizeof(unsigned long long)));
  bufs.p[3] = d_cnt;
  // FP64 basis of the list (for a group: of every dataset, D regions per
  // array), then for a group the D x list value matrix and the objective's
  // basis
  const size_t nb64 = group ? (size_t)3 * D + D + 3 : 3;
  CK(cudaMalloc(&b64, nb64 * lstride * sizeof(double)));
  bufs.p[4] = b64;
  CK(cudaMalloc(&table, tsize * sizeof(unsigned long long)));
  bufs.p[5] = table;
  CK(cudaMalloc(&d_lv, (size_t)levels * per_level));
  bufs.p[6] = d_lv;
  CK(cudaMemsetAsync(d_cnt, 0, (size_t)levels * sizeof(unsigned long long), s));
  auto rec_at = [&](int lv) { return (thoi_order_record*)(d_lv + (size_t)lv * per_level); };
  auto tops_at = [&](int lv) {
    return (TopEnt*)(d_lv + (size_t)lv * per_level + sizeof(thoi_order_record));
  };
  double* V = b64 + (group ? (size_t)3 * D : 3) * lstride;
  double* gb = V + (size_t)D * lstride;
  int launches = 0;
  // a group evaluates the candidates of every dataset in one batched FP64
  // launch: dataset descriptors, one slot per (order, dataset) with its own
  // region of the replicated list and of the basis, and per-slot counters
  struct GBufs {
    void* p = nullptr;
    ~GBufs() {
      if (p) cudaFree(p);
    }
  } gbuf;
  BatchDataset* d_ds = nullptr;
  BatchSlot* d_slots = nullptr;
  unsigned long long* ids_rep = nullptr;
  unsigned long long* counts_rep = nullptr;
  if (group) {
    std::vector<BatchDataset> hds(D);
    std::vector<BatchSlot> hsl((size_t)levels * D);
    for (int d = 0; d < D; d++) {
      hds[d].R32 = ctxs[d]->R32;
      hds[d].R64 = ctxs[d]->R64;
      hds[d].ls = ctxs[d]->ls;
      hds[d].N = N;
      hds[d].tau_piv = ctxs[d]->opt.pivot_tau;
      hds[d].tau_tr = ctxs[d]->opt.trace_tau;
      hds[d].pad = 0;
      for (int lv = 0; lv < levels; lv++) {
        BatchSlot& b = hsl[(size_t)lv * D + d];
        memset(&b, 0, sizeof b);
        b.d = d;
        b.k = k0 + lv;
        b.n = binom_host(N, k0 + lv);
        b.id_base = 0;
        b.flag_off = (unsigned long long)d * lstride;
        b.flag_cap = cap;
        b.cmb = combine_for(ctxs[d], k0 + lv);
      }
    }
    const size_t bytes = hds.size() * sizeof(BatchDataset) + hsl.size() * sizeof(BatchSlot) +
                         (size_t)D * lstride * 8 + (size_t)levels * D * 8;
    CK(cudaMalloc(&gbuf.p, bytes));
    unsigned char* q = (unsigned char*)gbuf.p;
    d_ds = (BatchDataset*)q;
    d_slots = (BatchSlot*)(q + hds.size() * sizeof(BatchDataset));
    ids_rep = (unsigned long long*)(q + hds.size() * sizeof(BatchDataset) +
                                    hsl.size() * sizeof(BatchSlot));
    counts_rep = ids_rep + (size_t)D * lstride;
    CK(cudaMemcpyAsync(d_ds, hds.data(), hds.size() * sizeof(BatchDataset),
                       cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_slots, hsl.data(), hsl.size() * sizeof(BatchSlot),
                       cudaMemcpyHostToDevice, s));
  }
  // order k0: exhaustive
  {
    const int32_t ord = k0;
    int nl = 0;
    if (group) {
      uint64_t ev = 0;
      st = enqueue_group(ctxs, D, &ord, 1, 0, binom_host(N, k0), measure, objective,
                         THOI_RED_PER_ORDER, nullptr, rec_at(0), tops_at(0), gstatus, gnref, s,
                         &nl, &ev);
    } else {
      st = enqueue_measures(c, &ord, 1, 0, binom_host(N, k0), THOI_RED_PER_ORDER, nullptr,
                            rec_at(0), tops_at(0), s, &nl, false, sel);
    }
    if (st != THOI_OK) return st;
    launches += nl;
  }
  // orders k0+1 .. k1: expansion of the selection, on the device
  int red_blocks = (int)(cap / 4096) + 1;  // few candidates: a few blocks, few lists to merge
  if (red_blocks > ref_cap) red_blocks = ref_cap;
  if (sel) {
    st = ensure_sel_ws(c);
    if (st != THOI_OK) return st;
  }
  for (int k = k0 + 1; k <= k1; k++) {
    const int lv = k - k0;
    unsigned long long* cnt = d_cnt + lv;
    CK(cudaMemsetAsync(table, 0, tsize * sizeof(unsigned long long), s));
    CK(launch_greedy_expand(rec_at(lv - 1), tops_at(lv - 1) + (size_t)side * kappa, kappa, N,
                            k - 1, c->binom, table, tsize, d_ids, cnt, s));
    launches++;
    SlotRange r;
    r.k = k;
    r.off = 0;
    r.r0 = 0;
    r.r1 = binom_host(N, k);
    Combine rc = group_combine();
    const double* rb = b64;
    if (!group) {
      NpletArgs a = base_args(c, r);
      a.mode = 2;
      a.flag_ids = d_ids;
      a.flag_count = cnt;
      a.flag_cap = cap;
      int grid = 0;
      CK(launch_nplet_f64s(a, true, b64, lstride, c->num_sms, s, &grid,
                           c->num_sms * MAX_BLOCKS_PER_SM_OUT));
      launches++;
      rc = a.cmb;
    } else {
      // every dataset in one launch: the list replicated per slot, the batched
      // FP64 kernel (grid.y = dataset), one measure per dataset, the objective
      const BatchSlot* sl = d_slots + (size_t)lv * D;
      unsigned long long* cr = counts_rep + (size_t)lv * D;
      const unsigned long long bstride = (unsigned long long)D * lstride;
      int bx = 2 * c->num_sms / D;
      if (bx < 1) bx = 1;
      if (bx > 64) bx = 64;
      CK(launch_group_replicate(d_ids, cnt, cap, D, lstride, ids_rep, cr, s));
      CK(launch_refactor_batch(d_ds, sl, 0, D, N, k, N > 32, c->binom, ids_rep, cr, b64, bstride,
                               gstatus, bx, s));
      CK(launch_group_pick_batch(b64, bstride, lstride, D, sl, cnt, cap, measure, V, s));
      CK(launch_group_combine(V, lstride, cap, cnt, D, objective, nullptr, gb, lstride,
                              c->num_sms, s));
      launches += 4;
      rb = gb;
    }
    int grid = 0;
    if (sel) {
      CK(launch_select_list64(rb, lstride, d_ids, cnt, cap, rc, kappa, c->sel_ws, c->status, part,
                              ptop, ref_cap, s, &grid));
      launches += sel_kernels(kappa) - 1;  // (one counted below)
    } else {
      CK(launch_reduce_list64(rb, lstride, d_ids, cnt, cap, rc, kappa, part, ptop, c->num_sms,
                              red_blocks, s, &grid));
    }
    MergeDescs MD;
    memset(&MD, 0, sizeof MD);
    MD.d[0].p32_off = 0;
    MD.d[0].g32 = grid;
    MD.d[0].k = k;
    MD.d[0].cmb = rc;
    CK(launch_merge(MD, 1, part, ptop, part, ptop, kappa, rec_at(lv), tops_at(lv), s));
    launches += 2;
  }
  // every order's selection, read once
  std::vector<unsigned char> host((size_t)levels * per_level);
  std::vector<unsigned long long> counts(levels);
  CK(cudaMemcpyAsync(host.data(), d_lv, host.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(counts.data(), d_cnt, (size_t)levels * 8, cudaMemcpyDeviceToHost, s));
  int hs = 0;
  for (int d = 0; d < D; d++) {
    int h = 0;
    CK(cudaMemcpyAsync(&h, ctxs[d]->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    hs |= h;
  }
  if (group) {
    int h = 0;
    CK(cudaMemcpyAsync(&h, gstatus, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    hs |= h;
  }
  CK(cudaStreamSynchronize(s));
  if (sel && (hs & ST_INEXACT) && !(hs & ST_CANCELLED))
    return greedy_impl(ctxs, D, objective, k0, k1, kappa, measure, maximize, sets_out, values_out,
                       stats, s, false);
  uint64_t evaluated = binom_host(N, k0);
  for (int lv = 0; lv < levels; lv++) {
    const int k = k0 + lv;
    const thoi_order_record* R = (const thoi_order_record*)(host.data() + (size_t)lv * per_level);
    const thoi_top_entry* T =
        (const thoi_top_entry*)(host.data() + (size_t)lv * per_level + sizeof(thoi_order_record)) +
        (size_t)side * kappa;
    const int n = R->top_count < kappa ? R->top_count : kappa;
    for (int i = 0; i < n; i++) {
      sets_out[(size_t)lv * kappa + i] = rank_to_mask(N, k, T[i].id);
      values_out[(size_t)lv * kappa + i] = T[i].value;
    }
    if (lv > 0) evaluated += counts[lv];
  }
  if (stats) {
    memset(stats, 0, sizeof *stats);
    stats->nplets = evaluated * (uint64_t)D;
    stats->launches = launches;
  }
  if (hs & ST_CANCELLED) return THOI_ERR_CANCELLED;
  return THOI_OK;  // candidates that are not positive definite are left out, not fatal
}

extern "C" thoi_status thoi_greedy(thoi_ctx* c, int32_t k0, int32_t k1, int32_t kappa,
                                   int32_t measure, int32_t maximize, uint64_t* sets_out,
                                   double* values_out, thoi_stats* stats, void* stream) {
  if (!c || !sets_out || !values_out || k0 < 1 || k1 < k0 || k1 > c->N || kappa < 1 ||
      kappa > THOI_MAX_TOP_M || measure < THOI_H || measure > THOI_S)
    return THOI_ERR_INVALID_ARG;
  return greedy_impl(&c, 1, -1, k0, k1, kappa, measure, maximize, sets_out, values_out, stats,
                     (cudaStream_t)stream);
}

extern "C" thoi_status thoi_group_greedy(thoi_ctx* const* ctxs, int32_t D, int32_t k0, int32_t k1,
                                         int32_t kappa, int32_t measure, int32_t objective,
                                         int32_t maximize, uint64_t* sets_out, double* values_out,
                                         thoi_stats* stats, void* stream) {
  thoi_status st = group_args_ok(ctxs, D, measure, objective);
  if (st != THOI_OK) return st;
  if (!sets_out || !values_out || k0 < 1 || k1 < k0 || k1 > ctxs[0]->N || kappa < 1 ||
      kappa > THOI_MAX_TOP_M)
    return THOI_ERR_INVALID_ARG;
  return greedy_impl(ctxs, D, objective, k0, k1, kappa, measure, maximize, sets_out, values_out,
                     stats, (cudaStream_t)stream);
}

// ------------------------------------------------------------------ API: simulated annealing
// Simulated annealing on one context's measure (D = 1) or on a group
// objective over D contexts.
static thoi_status anneal_impl(thoi_ctx* const* ctxs, int D, int objective, int32_t k_lo,
                               int32_t k_hi, int32_t n_chains, int32_t iters, double T0,
                               double alpha, int32_t patience, int32_t measure, int32_t maximize, uint64_t seed,
                               uint64_t* final_masks, double* final_values, uint64_t* best_masks,
                               double* best_values, thoi_stats* stats, cudaStream_t s) {
  const int nc = k_hi + 1;
  // host staging: combine tables (D x nc), then the R and log-variance pointers
  std::vector<Combine> tab((size_t)D * nc);
  std::vector<const double*> ptrs(2 * (size_t)D);
  for (int d = 0; d < D; d++) {
    for (int k = 0; k < nc; k++) tab[(size_t)d * nc + k] = combine_for(ctxs[d], k);
    ptrs[d] = ctxs[d]->R64;
    ptrs[D + d] = ctxs[d]->ls;
  }
  struct Bufs {
    void* p = nullptr;
    ~Bufs() {
      if (p) cudaFree(p);
    }
  } buf;
  const size_t n = (size_t)n_chains;
  const size_t tab_bytes = tab.size() * sizeof(Combine), ptr_bytes = ptrs.size() * sizeof(void*);
  const size_t bytes = tab_bytes + ptr_bytes + n * (4 * 8 + 8);
  CK(cudaMalloc(&buf.p, bytes));
  unsigned char* base = (unsigned char*)buf.p;
  Combine* d_tab = (Combine*)base;
  const double** d_ptrs = (const double**)(base + tab_bytes);
  unsigned long long* fm = (unsigned long long*)(base + tab_bytes + ptr_bytes);
  double* fv = (double*)(fm + n);
  unsigned long long* bm = (unsigned long long*)(fv + n);
  double* bv = (double*)(bm + n);
  unsigned long long* acc = (unsigned long long*)(bv + n);
  CK(cudaMemcpyAsync(d_tab, tab.data(), tab_bytes, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_ptrs, ptrs.data(), ptr_bytes, cudaMemcpyHostToDevice, s));
  CK(launch_anneal(d_ptrs, d_ptrs + D, D, objective, ctxs[0]->N, k_lo, k_hi, d_tab,
                   ctxs[0]->R64, ctxs[0]->ls, n_chains, iters, T0, alpha, patience, measure,
                   maximize, seed,
                   fm, fv, bm, bv, acc, s));
  CK(cudaMemcpyAsync(final_masks, fm, n * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(final_values, fv, n * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(best_masks, bm, n * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(best_values, bv, n * 8, cudaMemcpyDeviceToHost, s));
  std::vector<unsigned long long> hacc(n);
  CK(cudaMemcpyAsync(hacc.data(), acc, n * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (stats) {
    memset(stats, 0, sizeof *stats);
    stats->nplets = (uint64_t)n * (uint64_t)(iters + 1) * (uint64_t)D;  // evaluations
    unsigned long long a = 0;
    for (auto x : hacc) a += x;
    stats->n_refactored = a;  // accepted moves (these entry points evaluate in FP64 only)
    stats->launches = 1;
  }
  return THOI_OK;
}

static bool anneal_args_ok(int N, int32_t k_lo, int32_t k_hi, int32_t n_chains, int32_t iters,
                           double T0, double alpha, int32_t patience, int32_t measure, const void* a, const void* b,
                           const void* c, const void* d) {
  return k_lo >= 1 && k_hi >= k_lo && k_hi <= N && k_hi <= 32 && n_chains >= 1 && iters >= 0 &&
         T0 > 0.0 && alpha > 0.0 && patience >= 0 && measure >= THOI_H && measure <= THOI_S && a && b && c && d;
}

extern "C" thoi_status thoi_anneal(thoi_ctx* c, int32_t k_lo, int32_t k_hi, int32_t n_chains,
                                   int32_t iters, double T0, double alpha, int32_t patience,
                                   int32_t measure, int32_t maximize, uint64_t seed,
                                   uint64_t* final_masks, double* final_values,
                                   uint64_t* best_masks, double* best_values, thoi_stats* stats,
                                   void* stream) {
  if (!c || !anneal_args_ok(c->N, k_lo, k_hi, n_chains, iters, T0, alpha, patience, measure,
                            final_masks, final_values, best_masks, best_values))
    return THOI_ERR_INVALID_ARG;
  return anneal_impl(&c, 1, -1, k_lo, k_hi, n_chains, iters, T0, alpha, patience, measure,
                     maximize, seed, final_masks, final_values, best_masks, best_values, stats,
                     (cudaStream_t)stream);
}

extern "C" thoi_status thoi_group_anneal(thoi_ctx* const* ctxs, int32_t D, int32_t k_lo,
                                         int32_t k_hi, int32_t n_chains, int32_t iters, double T0,
                                         double alpha, int32_t patience, int32_t measure,
                                         int32_t objective, int32_t maximize, uint64_t seed,
                                         uint64_t* final_masks, double* final_values,
                                         uint64_t* best_masks, double* best_values,
                                         thoi_stats* stats, void* stream) {
  thoi_status st = group_args_ok(ctxs, D, measure, objective);
  if (st != THOI_OK) return st;
  if (!anneal_args_ok(ctxs[0]->N, k_lo, k_hi, n_chains, iters, T0, alpha, patience, measure,
                      final_masks, final_values, best_masks, best_values))
    return THOI_ERR_INVALID_ARG;
  return anneal_impl(ctxs, D, objective, k_lo, k_hi, n_chains, iters, T0, alpha, patience,
                     measure, maximize, seed, final_masks, final_values, best_masks, best_values,
                     stats, (cudaStream_t)stream);
}

// ------------------------------------------------------------------ API: autotune
static void tune_load(const char* path, const char* gpu, int sms) {
  FILE* f = fopen(path, "r");
  if (!f) return;
  char line[1024];
  while (fgets(line, sizeof line, f)) {
    char g[256] = {0};
    int sm = 0, k = 0, wide = 0, lanes = 0, chunk = 0, bps = 0;
    const char* q = strstr(line, "\"gpu\": \"");
    if (!q) continue;
    q += 8;
    int n = 0;
    while (q[n] && q[n] != '"' && n < 255) { g[n] = q[n]; n++; }
    if (sscanf(strstr(line, "\"sms\""), "\"sms\": %d, \"k\": %d, \"wide\": %d, \"lanes\": %d, "
                                          "\"chunk\": %d, \"blocks_per_sm\": %d",
               &sm, &k, &wide, &lanes, &chunk, &bps) != 6)
      continue;
    if (strcmp(g, gpu) != 0 || sm != sms || !shape_available(k, lanes)) continue;
    int prefix = 0;
    const char* pq = strstr(line, "\"prefix\"");
    if (pq && sscanf(pq, "\"prefix\": %d", &prefix) != 1) prefix = 0;
    // "out": the use the shape was tuned for; an entry without it (a shape
    // written by hand) serves both uses
    int out = -1;
    const char* oq = strstr(line, "\"out\"");
    if (oq && sscanf(oq, "\"out\": %d", &out) != 1) out = -1;
    Shape sh;
    sh.lanes = lanes;
    sh.chunk = chunk;
    sh.blocks_per_sm = bps;
    sh.prefix = (prefix >= 0 && prefix <= 5) ? prefix : 0;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (out != 1) g_tune[tune_key(gpu, sms, k, wide, 0)] = sh;
    if (out != 0) g_tune[tune_key(gpu, sms, k, wide, 1)] = sh;
    g_tune_gen++;
  }
  fclose(f);
}

static void tune_save(const char* path, const char* gpu, int sms) {
  FILE* f = fopen(path, "w");
  if (!f) return;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  fprintf(f, "[\n");
  bool first = true;
  for (auto& kv : g_tune) {
    char g[256];
    int sm, k, wide, out;
    if (sscanf(kv.first.c_str(), "%255[^|]|%d|%d|%d|%d", g, &sm, &k, &wide, &out) != 5) continue;
    if (strcmp(g, gpu) != 0 || sm != sms) continue;
    fprintf(f, "%s{\"gpu\": \"%s\", \"sms\": %d, \"k\": %d, \"wide\": %d, \"lanes\": %d, "
               "\"chunk\": %d, \"blocks_per_sm\": %d, \"prefix\": %d, \"out\": %d}",
            first ? "" : ",\n", g, sm, k, wide, kv.second.lanes, kv.second.chunk,
            kv.second.blocks_per_sm, kv.second.prefix, out);
    first = false;
  }
  fprintf(f, "\n]\n");
  fclose(f);
}

// Time the FP32 nplet kernel of order k with shape sh on the first n nplets
// (CUDA events on `s`), reducing to records, or with out (device, room for
// the n nplets' five measures) storing every nplet's measures; returns
// milliseconds or a negative value on error.
static double time_shape(thoi_ctx* c, int k, uint64_t n, const Shape& sh, cudaStream_t s,
                         void* out = nullptr) {
  const int saved_profile = c->opt.profile;
  c->opt.profile = 1;
  c->force_shape = sh;
  c->force_shape_valid = 1;
  double best = -1.0;
  const size_t need = thoi_records_bytes(1, c->opt.top_m);
  if (grow(&c->rec_buf, &c->rec_cap, need) == THOI_OK) {
    thoi_order_record* recs = (thoi_order_record*)c->rec_buf;
    TopEnt* tops = (TopEnt*)(c->rec_buf + sizeof(thoi_order_record));
    const int32_t ord = k;
    for (int rep = 0; rep < 3; rep++) {
      int launches = 0;
      thoi_stats st;
      const thoi_status es =
          out ? enqueue_measures(c, &ord, 1, 0, n, THOI_RED_NONE, out, nullptr, nullptr, s,
                                 &launches)
              : enqueue_measures(c, &ord, 1, 0, n, THOI_RED_PER_ORDER, nullptr, recs, tops, s,
                                 &launches, true);
      if (es != THOI_OK) break;
      const thoi_status fs = finish_status(c, s, 1, &st, n, launches);
      if (fs != THOI_OK && fs != THOI_ERR_NOT_PD) break;
      if (rep > 0 && (best < 0 || st.nplet_ms < best)) best = st.nplet_ms;  // rep 0 warms up
    }
  }
  c->force_shape_valid = 0;
  c->opt.profile = saved_profile;
  return best;
}

extern "C" thoi_status thoi_autotune(thoi_ctx* c, int32_t kmin, int32_t kmax, const char* cache_path,
                                     void* stream) {
  if (!c || kmin < 1 || kmax < kmin || kmax > c->N) return THOI_ERR_INVALID_ARG;
  if (c->opt.precision != THOI_F32_FIX64) return THOI_OK;  // only the FP32 kernels have shapes
  cudaStream_t s = (cudaStream_t)stream;
  if (cache_path) tune_load(cache_path, c->gpu_name, c->num_sms);
  const int wide = c->N > 32;
  void* ob = nullptr;  // output buffer for timing per-nplet output
  size_t ob_cap = 0;
  for (int k = kmin; k <= kmax; k++) {
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      if (g_tune.count(tune_key(c->gpu_name, c->num_sms, k, wide, 0))) continue;
    }
    const uint64_t total = binom_host(c->N, k);
    if (total < (1ull << 17)) continue;  // too small to matter: built-in shape
    // where the prefix-shared kernel competes, every candidate is timed on
    // the whole order (that kernel covers whole orders only); elsewhere on the
    // first 2^22 nplets, scaled to the order
    const bool pfx_candidate = k >= KPFX_MIN && k <= KPFX2_MAX && total <= (1ull << 28);
    const uint64_t n = pfx_candidate ? total : (total < (1ull << 22) ? total : (1ull << 22));
    Shape best = default_shape(k);
    double best_ms = -1.0;
    for (int lanes = 1; lanes <= 4; lanes <<= 1) {
      if (!shape_available(k, lanes)) continue;
      // above the one-thread register kernels, lanes = 1 is the generic
      // kernel: never faster than a lane group
      if (lanes == 1 && k > KREG_MAX && (shape_available(k, 2) || shape_available(k, 4))) continue;
      for (int chunk = 4; chunk <= 8; chunk <<= 1) {
        Shape sh;
        sh.lanes = lanes;
        sh.chunk = chunk;
        sh.blocks_per_sm = 0;
        sh.prefix = 0;
        const double ms = time_shape(c, k, n, sh, s) * (double)total / (double)n;
        if (ms > 0 && (best_ms < 0 || ms < best_ms)) {
          best_ms = ms;
          best = sh;
        }
      }
    }
    const Shape best_dense = best;
    Shape best_pfx = best;
    double pfx_ms = -1.0;
    // the prefix-shared kernel covers whole orders: timed on the whole order
    // when that is affordable (up to 2^28 nplets)
    if (pfx_candidate) {
      // (k-1)-prefix kernel with 1, 2, 4 prefixes per thread per round, then
      // the (k-2)-prefix kernel with 1, 2, then that kernel with the last
      // variables two at a time, with 1, 2, then (from order 5) the
      // three-level and (from order 6) the four-level kernel with the last
      // variables two at a time, with 1, 2
      for (int v = 0; v < 11; v++) {
        if ((v >= 7 && k < 5) || (v >= 9 && k < 6)) break;
        if (v < 3 && k > KPFX_MAX) continue;  // the one-level kernel stops at KPFX_MAX
        Shape sh;
        sh.lanes = 1;
        sh.chunk = v < 3 ? 1 << v : 1 << ((v - 3) & 1);
        sh.blocks_per_sm = 0;
        sh.prefix = v < 3 ? 1 : (v < 5 ? 2 : (v < 7 ? 3 : (v < 9 ? 4 : 5)));
        const double ms = time_shape(c, k, total, sh, s);
        if (ms > 0 && (pfx_ms < 0 || ms < pfx_ms)) {
          pfx_ms = ms;
          best_pfx = sh;
        }
        if (ms > 0 && (best_ms < 0 || ms < best_ms)) {
          best_ms = ms;
          best = sh;
        }
      }
    }
    // per-nplet output: the best dense and the best prefix shape timed again
    // storing every nplet's measures (the prefix kernels' stores are
    // scattered); the dense shape where no prefix shape ran or the output
    // buffer cannot be had
    Shape best_out = best_dense;
    if (pfx_ms > 0) {
      const size_t ob_need = (size_t)5 * total * (c->opt.out_f64 ? 8 : 4);
      if (ob_need > ob_cap) {
        if (ob) cudaFree(ob);
        ob = nullptr;
        ob_cap = 0;
        if (cudaMalloc(&ob, ob_need) == cudaSuccess) {
          ob_cap = ob_need;
        } else {
          ob = nullptr;
          cudaGetLastError();
        }
      }
      if (ob) {
        const double md = time_shape(c, k, total, best_dense, s, ob);
        const double mp = time_shape(c, k, total, best_pfx, s, ob);
        if (mp > 0 && (md < 0 || mp < md)) best_out = best_pfx;
      }
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[tune_key(c->gpu_name, c->num_sms, k, wide, 0)] = best;
    g_tune[tune_key(c->gpu_name, c->num_sms, k, wide, 1)] = best_out;
    g_tune_gen++;
  }
  if (ob) cudaFree(ob);
  if (cache_path) tune_save(cache_path, c->gpu_name, c->num_sms);
  return THOI_OK;
}
