/*
 * thoi.h -- C ABI of the GB300 library for exhaustive Gaussian-copula
 * higher-order information (arXiv 2501.03381, "THOI").
 *
 * Given a T x N sample matrix, the library estimates the Gaussian-copula
 * covariance (Supp. eq. gaussian_copula_covariance_estimator) on the GPU and
 * evaluates, for every subset ("nplet") of k of the N variables, the joint
 * entropy H (Supp. eq. gaussian_differential_entropy), the total correlation
 * TC (eq. TC), the dual total correlation DTC (eq. DTC), the O-information
 * O = TC - DTC (eq. O-info) and the S-information S = TC + DTC (eq. S-info).
 * All entropies are in nats.
 *
 * Conventions shared by every entry point
 *  - Pointers are plain host or device pointers; the header needs no CUDA
 *    headers.  `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  Device pointers must belong to the current device.
 *  - Ownership: the caller owns X, every output buffer and the stream.  The
 *    context owns its covariance copies, tables and workspace and frees them
 *    in thoi_destroy().
 *  - Ordering: work is queued on `stream`; calls return once it is queued
 *    unless stated otherwise.  Argument errors are returned immediately.
 *    Errors found on the device (a non-positive-definite nplet, a workspace
 *    overflow) are returned by the call that synchronises (thoi_create and
 *    the record/grad entry points read a status word back before returning).
 *  - Threads: a context may be used by one host thread at a time.  The only
 *    global state is the autotuner cache, guarded by a mutex.
 *  - Enumeration (Supp. eq. comb): the requested orders are visited in the
 *    caller's order; within an order, k-subsets c_0 < ... < c_{k-1} come in
 *    lexicographic order.  The global id of a nplet is its position in that
 *    sequence (order offset + lexicographic rank).
 */
#ifndef THOI_API_H_
#define THOI_API_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define THOI_MAX_N 64      /* largest number of variables */
#define THOI_MAX_TOP_M 1024 /* largest top-M list per order and side */
#define THOI_MAX_GROUP 1024 /* largest number of datasets in a group objective */

typedef struct thoi_ctx thoi_ctx;

typedef enum {
  THOI_OK = 0,
  THOI_ERR_INVALID_ARG = 1,     /* bad size, order, pointer or option */
  THOI_ERR_NONFINITE_INPUT = 2, /* X holds NaN or Inf */
  THOI_ERR_TOO_LARGE = 3,       /* N > THOI_MAX_N, or a size beyond a documented limit */
  THOI_ERR_NOT_PD = 4,          /* some nplet is not positive definite even in FP64;
                                   its measures are NaN and it is left out of reductions */
  THOI_ERR_OOM = 5,             /* a device allocation failed */
  THOI_ERR_CUDA = 6,            /* a CUDA runtime call failed */
  THOI_ERR_TIMEOUT = 7,         /* a bounded device wait gave up */
  THOI_ERR_CANCELLED = 8,       /* the cancel flag was raised */
  THOI_ERR_WORKSPACE = 9        /* more flagged nplets than the re-factor list holds */
} thoi_status;

typedef enum {
  THOI_F32_FIX64 = 0, /* FP32 Cholesky; flagged nplets re-factored in FP64 */
  THOI_F64 = 1        /* every nplet in FP64 */
} thoi_precision;

typedef enum {
  THOI_RED_NONE = 0,     /* per-nplet SoA output */
  THOI_RED_PER_ORDER = 1 /* per-order reduction records */
} thoi_reduction_kind;

typedef enum { THOI_DTYPE_F32 = 0, THOI_DTYPE_F64 = 1 } thoi_dtype;

typedef enum { THOI_H = 0, THOI_TC = 1, THOI_DTC = 2, THOI_O = 3, THOI_S = 4 } thoi_measure;

/* Group objectives over D datasets (see thoi_group_measures). */
typedef enum {
  THOI_GROUP_MEAN = 0,    /* mean of the measure over the datasets */
  THOI_GROUP_COHEN_D = 1  /* paired Cohen's d between two conditions */
} thoi_group_objective;

typedef enum {
  THOI_SIGMA32_TENSORCORE = 0, /* split-BF16 tensor-core GEMM, FP32 accumulation */
  THOI_SIGMA32_FROM_F64 = 1    /* FP32 rounding of the FP64 covariance */
} thoi_sigma32_source;

/* How the FP32 path forms per-order records (thoi_measures with
 * THOI_RED_PER_ORDER).  Fused: the nplet kernels keep the sums and the count
 * of O < 0 per thread and list only the nplets beyond bounds taken from a
 * sample of the order, so no per-nplet value reaches device memory; the
 * merge certifies every extreme and top list against the bounds, and an
 * uncertified record repeats the request with stored values (the result is
 * the same either way).  Stored: every nplet's three basis values are
 * written and reduced by a streaming kernel. */
typedef enum {
  THOI_RECORDS_AUTO = 0,   /* fused for orders of at least 2^20 nplets (k <= 32), else stored */
  THOI_RECORDS_FUSED = 1,  /* fused for every order with k <= 32 */
  THOI_RECORDS_STORED = 2  /* always stored basis values */
} thoi_records_mode;

/* Options; fill with thoi_default_options() and change what you need. */
typedef struct {
  int32_t precision;     /* thoi_precision; default THOI_F32_FIX64 */
  float pivot_tau;       /* re-factor a nplet in FP64 when its smallest Cholesky pivot
                            of the correlation submatrix is below this; default 1e-2 */
  float trace_tau;       /* ... or when trace((R_S)^-1) exceeds this; default 100 */
  int32_t bias_correct;  /* subtract the Gaussian entropy bias (Supp. eq. bias_corrector,
                            with 1/2 on the digamma sum) from every entropy; default 0 */
  int32_t top_m;         /* length of the top-M lists by O per order and side, 0..1024;
                            default 256 */
  int32_t out_f64;       /* per-nplet output in FP64 (1) or FP32 (0); default: 1 for
                            THOI_F64, 0 otherwise */
  int32_t sigma32_source;/* thoi_sigma32_source; default THOI_SIGMA32_FROM_F64 (the
                            tensor-core GEMM is about 1e-7 relative off, which moves O
                            by up to ~1e-4 at k >= 20 on ill-conditioned nplets) */
  int32_t autotune;      /* use the autotuner's launch shapes (1) or the built-in ones (0);
                            default 1 */
  uint64_t flag_capacity;/* entries of the FP64 re-factor list; 0 = automatic */
  int32_t profile;       /* 1: time the kernels with CUDA events on `stream` and report
                            the times in thoi_stats; default 0 */
  int32_t records_mode;  /* thoi_records_mode; default THOI_RECORDS_AUTO */
} thoi_options;

/* Per-order reduction record (Fig. 1A caption: a function applied to every
 * batch, e.g. the minimum O, read as this fixed set).  Measures are indexed
 * by thoi_measure.  Ties in min/max go to the smallest global id.  Nplets
 * that are not positive definite are counted in n_not_pd and left out. */
typedef struct {
  int32_t k;
  int32_t top_count;     /* valid entries in each top list (min(top_m, count)) */
  uint64_t count;        /* nplets of order k inside [id_begin, id_end) */
  uint64_t count_neg_O;  /* nplets with O < 0 */
  uint64_t n_refactored; /* nplets re-computed in FP64 (FP32 path) */
  uint64_t n_not_pd;     /* nplets not positive definite in FP64 either */
  double min[5];
  double max[5];
  double mean[5];
  uint64_t argmin[5];    /* global ids */
  uint64_t argmax[5];
} thoi_order_record;

/* One top-M entry: value of O and global id. */
typedef struct {
  double value;
  uint64_t id;
} thoi_top_entry;

/* Statistics of the last thoi_measures call (filled after it synchronises). */
typedef struct {
  uint64_t nplets;       /* nplets evaluated */
  uint64_t n_refactored; /* nplets re-computed in FP64 */
  uint64_t n_not_pd;     /* nplets not positive definite */
  int32_t launches;      /* kernel launches queued by the call */
  int32_t nplet_launches;/* thoi_batch_measures: launches of the batched nplet kernel
                            (one per band of orders: 1..8, 9..14, 15..17, 18..20) */
  /* device time in milliseconds, measured with CUDA events when opt.profile = 1
     (otherwise 0): the nplet kernels (FP32 or FP64 path), the FP64 re-factor
     kernels, the merge, and the streaming reduction */
  double nplet_ms;
  double refactor_ms;
  double merge_ms;
  double reduce_ms;      /* the per-order reduction kernels of the FP32 path (streaming
                            reduction, or the sample bounds and candidate list of
                            fused records) */
  int32_t fused_retries; /* 1 when fused records could not be certified and the
                            request was repeated with stored values */
  int32_t pad2;
  uint64_t n_candidates; /* fused records: nplets listed beyond the sample bounds */
} thoi_stats;

/* Fill `opt` with the defaults listed above. */
void thoi_default_options(thoi_options* opt);

/* Create a context from a T x N sample matrix (rows = samples).
 *  X      : host or device pointer (detected), element (t, i) at X[t*ld + i]
 *  T, N   : samples and variables, 2 <= N <= THOI_MAX_N, T >= N + 1, T <= 2^24
 *  ld     : leading dimension in elements, ld >= N
 *  dtype  : thoi_dtype of X
 *  opt    : options (NULL = defaults)
 * Runs the copula transform (per-column ordinal rank with ties broken by
 * sample index, u = (r+1)/(T+1), z = Phi^{-1}(u)) and the covariance (centred,
 * divided by T-1) on the device (Supp. eq.
 * gaussian_copula_covariance_estimator), then synchronises `stream`.
 * Returns THOI_ERR_NONFINITE_INPUT when X holds NaN or Inf.  X may be freed
 * once the call returns. */
thoi_status thoi_create(thoi_ctx** out, const void* X, int64_t T, int64_t N, int64_t ld,
                        int32_t dtype, const thoi_options* opt, void* stream);

/* Create a context from an explicit N x N covariance (host or device,
 * row-major FP64): the Sigma the paper's estimators start from once the
 * copula covariance is known (Methods, "Efficient computation of HOI via
 * Gaussian copulas": the covariance is computed once and every entropy is a
 * function of its submatrices, Supp. eq. gaussian_differential_entropy).
 * Every diagonal entry must be positive and finite (THOI_ERR_INVALID_ARG
 * otherwise).  T_for_bias is the sample count used by the bias corrector
 * (Supp. eq. bias_corrector; ignored unless opt->bias_correct).  The caller
 * may free Sigma once the call returns; synchronises `stream`. */
thoi_status thoi_create_from_cov(thoi_ctx** out, const double* Sigma, int64_t N,
                                 int64_t T_for_bias, const thoi_options* opt, void* stream);

/* Copy the context's covariance out: Sigma64 (N x N FP64) and/or Sigma32
 * (N x N FP32, the matrix the FP32 path starts from); either may be NULL.
 * Host or device destinations; synchronises `stream`. */
thoi_status thoi_get_cov(thoi_ctx* ctx, double* Sigma64, float* Sigma32, void* stream);

/* Copy the per-column ordinal ranks (T x N int32, row-major) of the sample
 * matrix the context was created from (host or device destination).
 * THOI_ERR_INVALID_ARG for a context made by thoi_create_from_cov. */
thoi_status thoi_get_ranks(thoi_ctx* ctx, int32_t* ranks, void* stream);

/* Number of variables of the context. */
int64_t thoi_n(const thoi_ctx* ctx);

/* Exact number of nplets over the listed orders (host): the sum of the
 * binomial coefficients C(N, k) of Supp. eq. comb ("The combinatorial
 * explosion"), each exact in 64 bits for N <= 64.  An order outside 0..N
 * adds nothing; returns 0 for N outside 1..THOI_MAX_N, a null list or
 * n_orders < 1. */
uint64_t thoi_count(int64_t N, const int32_t* orders, int32_t n_orders);

/* Subset of a global id (host), in the enumeration order of Supp. eq. comb:
 * the id picks the order by the prefix sums of C(N, k) over the listed
 * orders, then the lexicographic rank r within order k gives the indices by
 * the combinatorial number system, r = C(N,k) - 1 - sum_i C(N-1-c_i, k-i).
 * Writes k indices c_0 < ... < c_{k-1} to idx_out (host, room for
 * THOI_MAX_N) and k to *k_out.  THOI_ERR_INVALID_ARG for an id beyond the
 * count, a bad order list or a null pointer. */
thoi_status thoi_unrank(int64_t N, const int32_t* orders, int32_t n_orders, uint64_t id,
                        int32_t* idx_out, int32_t* k_out);

/* Subsets of n global ids computed on the device with the kernels' own
 * unranking (combinatorial number system of Supp. eq. comb, as in
 * thoi_unrank) -- exposed so the enumeration can be checked.  ids: device u64[n]; idx_out: device int8[n * kmax], each row
 * holding the indices then -1 padding; kmax >= the largest listed order. */
thoi_status thoi_unrank_device(int64_t N, const int32_t* orders, int32_t n_orders,
                               const uint64_t* ids, int64_t n, int32_t kmax, int8_t* idx_out,
                               void* stream);

/* Bytes of the per-order record output for n_orders orders: the records,
 * then for each order its top-M largest O (descending) and top-M smallest O
 * (ascending), top_m thoi_top_entry each:
 *   [thoi_order_record x n_orders][thoi_top_entry x n_orders x 2 x top_m] */
size_t thoi_records_bytes(int32_t n_orders, int32_t top_m);

/* Evaluate the five measures of every nplet with global id in
 * [id_begin, id_end) (id_end = UINT64_MAX means all): H from Supp. eq.
 * gaussian_differential_entropy on the submatrix Sigma_S, and TC, DTC, O,
 * S from Methods eqs. TC, DTC, O-info, S-info, for all nplets in batches
 * (Methods, "Parallel and batched computation of HOI"); with
 * THOI_RED_PER_ORDER each order is reduced on the device instead of stored
 * (Fig. 1A caption: a function applied per batch, e.g. the minimum O).
 *  orders  : host int32[n_orders], each 1 <= k <= N
 *  kind    : THOI_RED_NONE -- `out` is a device array of 5 x n values (SoA,
 *            out[m * n + (id - id_begin)]), FP32 or FP64 per opt.out_f64;
 *            THOI_RED_PER_ORDER -- `out` is a host or device buffer of
 *            thoi_records_bytes(n_orders, top_m) bytes laid out as above.
 *  out_bytes : size of `out`, checked
 *  stats   : optional, filled after the call synchronises
 * The FP32 path factors each correlation submatrix R_S = L L^T in FP32 and
 * gets every leave-one-out log-determinant from log det R_S +
 * log (R_S^{-1})_jj; nplets whose smallest pivot is below pivot_tau, whose
 * trace(R_S^{-1}) exceeds trace_tau, or whose result is not finite are
 * re-factored in FP64.  The call synchronises `stream` before returning
 * (it reads the re-factor count back).  Returns THOI_ERR_NOT_PD when some
 * nplet is not positive definite in FP64. */
thoi_status thoi_measures(thoi_ctx* ctx, const int32_t* orders, int32_t n_orders,
                          uint64_t id_begin, uint64_t id_end, int32_t kind, void* out,
                          size_t out_bytes, thoi_stats* stats, void* stream);

/* Gradient of L = sum over every nplet of the listed orders of one measure
 * (thoi_measure) with respect to the covariance Sigma, its N^2 entries taken
 * as independent (the convention of d log det Sigma / d Sigma = Sigma^{-1}).
 * Per nplet with P = Sigma_S^{-1}, p_j = P_jj (from eq.
 * gaussian_differential_entropy):
 *   dO/dSigma_S = 1/2 [diag(1/Sigma_ii) - 2P + P diag(1/p) P]
 *   dS/dSigma_S = 1/2 [diag(1/Sigma_ii) - P diag(1/p) P]
 * (H, TC, DTC likewise), scattered into the N x N result.  dL_dSigma is a
 * device float[N*N] (row-major) owned by the caller.  The forward pass uses
 * the FP32 path with the FP64 re-factor; accumulation is in FP64.
 * Synchronises `stream`. */
thoi_status thoi_measures_grad(thoi_ctx* ctx, const int32_t* orders, int32_t n_orders,
                               int32_t measure, float* dL_dSigma, thoi_stats* stats,
                               void* stream);

/* Per-order reduction records for D contexts in one persistent launch per
 * order (the paper processes several datasets together, Methods "Parallel
 * and batched computation of HOI"; here they may differ in N and T).
 * Context d evaluates the orders kmin..min(kmax, N_d).  out is a host or
 * device buffer: for each context in turn, (kmax - kmin + 1) records then
 * their top lists, i.e. thoi_records_bytes(kmax - kmin + 1, top_m) bytes per
 * context (orders above N_d get count 0).  All contexts must use the same
 * precision and top_m.  The launches are captured once in a CUDA graph and
 * replayed.  Synchronises `stream`. */
thoi_status thoi_batch_measures(thoi_ctx* const* ctxs, int32_t D, int32_t kmin, int32_t kmax,
                                void* out, size_t out_bytes, thoi_stats* stats, void* stream);

/* Autotune the FP32 kernels' launch shapes for orders kmin..kmax on the
 * current GPU (timed on the device) and store the choice in the process-wide
 * cache; if cache_path is not NULL the cache is also written there as JSON
 * keyed by GPU name and SM count (and read from there first). */
thoi_status thoi_autotune(thoi_ctx* ctx, int32_t kmin, int32_t kmax, const char* cache_path,
                          void* stream);

/* Raise (1) or clear (0) the context's cancel flag; running and later
 * thoi_measures calls stop early and return THOI_ERR_CANCELLED. */
thoi_status thoi_set_cancel(thoi_ctx* ctx, int32_t flag);

/* Per-order reduction record of one order k, computed without allocating
 * any device memory (the paper has no counterpart; it exists for callers
 * that cannot call cudaMalloc or cudaFree -- for example a process whose
 * device memory budget is wholly held by another allocator, or one that
 * cannot afford the device-wide synchronisation those calls may cause).
 *  Sigma   : device pointer, N x N covariance, row-major FP64 (input)
 *  N, k    : 1 <= k <= N <= THOI_MAX_N and C(N, k) < 2^32
 *  top_m   : 0..16 entries per top list
 *  rec_out : device pointer to one thoi_order_record (output)
 *  top_out : device pointer to 2 * top_m thoi_top_entry (largest O
 *            descending, then smallest O ascending), or NULL when top_m = 0
 * Every nplet is evaluated in FP64 (the THOI_F64 path, no bias correction);
 * global ids are the lexicographic ranks within order k.  Scratch space
 * (1 MiB per device, held from library load until process exit) is one
 * static device array shared by all calls: calls whose work overlaps on the
 * GPU (different streams, or different host threads) race on it and must be
 * serialised by the caller.  Before it returns, the call queries pointer
 * attributes, copies the status word to host memory and synchronises
 * `stream`.  Sigma, rec_out and top_out must
 * be memory of the current device (THOI_ERR_INVALID_ARG otherwise).  Returns
 * THOI_ERR_TOO_LARGE for N > 64, top_m > 16 or C(N, k) >= 2^32; synchronises
 * `stream`; THOI_ERR_NOT_PD when a nplet is not positive definite. */
thoi_status thoi_order_record_noalloc(const double* Sigma, int64_t N, int32_t k, int32_t top_m,
                                      thoi_order_record* rec_out, thoi_top_entry* top_out,
                                      void* stream);

/* Greedy search (Methods, "Heuristics", "Greedy Algorithm").  Start from the
 * kappa best nplets of order k0 (an exhaustive pass over all C(N, k0)); then,
 * for each order k = k0+1 .. k1, grow every selected set by each variable it
 * lacks, evaluate the distinct candidates and keep the kappa best.  "Best" is
 * the largest (maximize != 0) or smallest value of `measure` (thoi_measure);
 * ties go to the smaller lexicographic rank.  All evaluations run in the FP64
 * path on the device, whatever the context's precision; candidates that are
 * not positive definite are left out.
 *  sets_out   : host uint64_t[(k1-k0+1) * kappa]; row k-k0 holds the selected
 *               sets of order k, best first, as bit masks (bit i = variable i)
 *  values_out : host double[(k1-k0+1) * kappa], the measure of each set
 * Unused slots (fewer than kappa candidates) hold mask 0 and NaN.
 * 1 <= k0 <= k1 <= N, 1 <= kappa <= THOI_MAX_TOP_M.  Synchronises `stream`. */
thoi_status thoi_greedy(thoi_ctx* ctx, int32_t k0, int32_t k1, int32_t kappa, int32_t measure,
                        int32_t maximize, uint64_t* sets_out, double* values_out,
                        thoi_stats* stats, void* stream);

/* Simulated annealing (Methods, "Heuristics", "Simulated Annealing
 * Algorithm").  n_chains independent chains, each a set of k_lo..k_hi
 * variables (k_hi <= 32), run on the device until one of the paper's two
 * termination criteria holds: `iters` steps done, or (patience > 0) no rise
 * of the chain's best energy over the last `patience` steps (the chain stops
 * after the first step t with t - t_best >= patience, t_best the last step
 * that raised the best energy, 0 at the start; patience = 0: off):
 *  - start: a random set (size uniform in k_lo..k_hi, members by a partial
 *    Fisher-Yates shuffle);
 *  - move: within one order (k_lo == k_hi) swap a member for a non-member;
 *    across orders add or remove a random variable while the size stays in
 *    range, else swap;
 *  - energy E = the measure (maximize != 0) or its negative, in FP64; sets
 *    that are not positive definite are rejected;
 *  - acceptance: always if E rises, else with probability exp(dE / Temp)
 *    (the usual Metropolis rule; the paper's printed exp(-dE / Temp) would
 *    accept every worse move);
 *  - cooling: Temp = T0 at step 1, multiplied by alpha after every step
 *    (step t runs at T0 * alpha^(t-1)).
 * Random numbers: draw (chain, step, slot) is the
 * ((chain * (iters+1) + step) * 64 + slot)-th output of SplitMix64 seeded with
 * `seed` (integers in [0, n): (z * n) >> 64; uniforms: (z >> 11) * 2^-53), so a
 * run is reproducible and checkable draw for draw.
 * Outputs (host, n_chains each): the final and the best set of every chain as
 * bit masks and their measure values.  stats->nplets = energies evaluated,
 * stats->n_refactored = accepted moves.  Synchronises `stream`. */
thoi_status thoi_anneal(thoi_ctx* ctx, int32_t k_lo, int32_t k_hi, int32_t n_chains, int32_t iters,
                        double T0, double alpha, int32_t patience, int32_t measure,
                        int32_t maximize, uint64_t seed,
                        uint64_t* final_masks, double* final_values, uint64_t* best_masks,
                        double* best_values, thoi_stats* stats, void* stream);

/* Group objective of one measure over D datasets, for every nplet (Results,
 * "Leveraging Gaussian entropy estimators with batch processing": the nplet
 * with the smallest average O across datasets; Methods, "fMRI analysis": the
 * paired Cohen's d between two conditions).  With v_d the measure of the
 * nplet in dataset d:
 *   THOI_GROUP_MEAN    : g = (1/D) sum_d v_d
 *   THOI_GROUP_COHEN_D : D = 2P, P >= 2; dataset i (condition A) is paired with
 *                        dataset P + i (condition B); delta_i = v_i - v_{P+i};
 *                        g = mean(delta) / sd(delta), sd with the P - 1
 *                        denominator
 * A nplet that is not positive definite in some dataset, or whose differences
 * all coincide (sd = 0), has no value: NaN per nplet, and in the records it is
 * left out and counted in n_not_pd.
 *  ctxs    : D contexts (1 <= D <= THOI_MAX_GROUP, 4 <= D even for Cohen's d)
 *            with the same N, all on the current device; a context may appear
 *            more than once.  Each
 *            dataset is evaluated by its own path (precision, thresholds,
 *            bias correction of its context); ctxs[0] holds the workspace
 *            and gives top_m.
 *  orders, id_begin, id_end : as in thoi_measures
 *  measure : thoi_measure the objective is taken of
 *  kind    : THOI_RED_NONE -- `out` is a device double[n], g of every nplet in
 *            [id_begin, id_end) in id order (out_bytes >= 8 n);
 *            THOI_RED_PER_ORDER -- `out` (host or device) receives the records
 *            in thoi_measures' layout, thoi_records_bytes(n_orders, top_m)
 *            bytes; every measure slot of a record carries g's minimum,
 *            maximum, mean and their ids, count_neg_O counts g < 0, the top
 *            lists rank g, and n_refactored sums the datasets' re-factors.
 * Device memory: ctxs[0] keeps a D x P_g matrix of FP64 values (at most
 * 16 GiB and a quarter of the free memory, P_g >= 65536), plus one FP64 basis
 * piece of P_g nplets; orders larger than P_g run in pieces.  stats: nplets =
 * evaluations (D per nplet), n_refactored summed over the datasets.
 * Statuses as in thoi_measures (THOI_ERR_NOT_PD when some nplet failed in
 * some dataset).  Synchronises `stream`. */
thoi_status thoi_group_measures(thoi_ctx* const* ctxs, int32_t D, const int32_t* orders,
                                int32_t n_orders, uint64_t id_begin, uint64_t id_end,
                                int32_t measure, int32_t objective, int32_t kind, void* out,
                                size_t out_bytes, thoi_stats* stats, void* stream);

/* Greedy search on a group objective (Methods, "Heuristics": the searches
 * take several datasets; Methods, "fMRI analysis": nplets that maximise or
 * minimise the paired Cohen's d).  As thoi_greedy, with "best" the largest
 * (maximize != 0) or smallest group objective g of `measure` over the D
 * contexts (thoi_group_measures); every evaluation in FP64.  Nplets without a
 * value are left out.  Same outputs and limits as thoi_greedy. */
thoi_status thoi_group_greedy(thoi_ctx* const* ctxs, int32_t D, int32_t k0, int32_t k1,
                              int32_t kappa, int32_t measure, int32_t objective,
                              int32_t maximize, uint64_t* sets_out, double* values_out,
                              thoi_stats* stats, void* stream);

/* Simulated annealing on a group objective: thoi_anneal with the energy
 * the group objective g (thoi_group_measures) of `measure` over the D
 * contexts, each set evaluated in FP64 in every dataset; sets without a
 * value are rejected.  Same draws, moves, outputs and limits as
 * thoi_anneal. */
thoi_status thoi_group_anneal(thoi_ctx* const* ctxs, int32_t D, int32_t k_lo, int32_t k_hi,
                              int32_t n_chains, int32_t iters, double T0, double alpha,
                              int32_t patience, int32_t measure, int32_t objective,
                              int32_t maximize,
                              uint64_t seed, uint64_t* final_masks, double* final_values,
                              uint64_t* best_masks, double* best_values, thoi_stats* stats,
                              void* stream);

/* Measured multiply-add peak of the CUDA cores of the current device (not part
 * of the method: it gives the roofline denominators of the FP32 nplet kernels
 * and of the FP64 re-factor).  fp64 = 0 times FFMA, fp64 = 1 DFMA: every
 * thread of a grid of 8 blocks of 256 threads per SM runs 8 independent
 * multiply-add chains of 16 * iters steps; the second of two launches is
 * timed with CUDA events on `stream`.  *tflops = 2 FLOP per multiply-add /
 * time; *ms (optional) = that launch's time.  Allocates a few KB; synchronises
 * `stream`.  THOI_ERR_INVALID_ARG for iters < 1 or a null tflops. */
thoi_status thoi_fma_peak(int32_t fp64, int32_t iters, double* tflops, double* ms, void* stream);

/* Host-only sharding helpers (no device work, no CUDA calls).  Nplets are
 * independent (Methods, "Parallel and batched computation of HOI"), so one
 * request splits into contiguous global-id ranges evaluated by separate
 * processes, one GPU each, whose per-order records are merged once.
 *
 * thoi_partition: bounds[0..R] (caller-owned, R + 1 entries) with bounds[0] = 0,
 * bounds[R] = thoi_count(N, orders, n_orders), non-decreasing, such that range
 * r = [bounds[r], bounds[r+1]) holds about 1/R of the work, a nplet of order
 * k weighing 2/3 k^3 + 2 k^2 (one LDL^T, one unit-lower inverse, the inverse
 * diagonal).  Exact integer arithmetic: the same bounds on every host.
 * THOI_ERR_INVALID_ARG for N outside 1..64, an order outside 1..N, R < 1 or a
 * null pointer. */
thoi_status thoi_partition(int64_t N, const int32_t* orders, int32_t n_orders, int32_t R,
                           uint64_t* bounds);

/* thoi_merge_records: merge R per-order record blocks produced for disjoint id
 * ranges of one request (same orders, same top_m).  in holds the R blocks back
 * to back, each thoi_records_bytes(n_orders, top_m) bytes in the layout
 * thoi_measures writes; out (caller-owned, one block) receives: counts summed,
 * min/max with the smallest id on ties, means weighted by the valid counts
 * (count - n_not_pd), and each top list re-selected from the union of the
 * ranks' lists by (value, id) (the union holds the global top-M, because
 * every global top-M entry is in its own range's top-M).  Host memory only.
 * THOI_ERR_INVALID_ARG when the blocks disagree on an order or an argument is
 * out of range. */
thoi_status thoi_merge_records(const void* in, int32_t R, int32_t n_orders, int32_t top_m,
                               void* out);

/* Human-readable name of a status. */
const char* thoi_status_string(thoi_status s);

/* Free the context and everything it owns. */
void thoi_destroy(thoi_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* THOI_API_H_ */
