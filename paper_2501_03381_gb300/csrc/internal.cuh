// Internal declarations shared by the library's CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "thoi.h"

namespace thoi {

constexpr int NB = THOI_MAX_N + 1;  // side of the binomial table C(n, m), n, m <= 64
constexpr int KREG_MAX = 24;        // largest order with a one-thread register FP32 kernel
constexpr int KBATCH_MAX = 20;      // largest order of the batched register kernel
constexpr int RED_NT = 128;         // threads per block of the nplet kernels
constexpr int TOP_CAP = 2048;       // top-M candidate buffer per side (power of two)

// Device status bits (OR-ed into the context's status word).
enum : int {
  ST_NOT_PD = 1,
  ST_FLAG_OVERFLOW = 2,
  ST_NONFINITE = 4,
  ST_CANCELLED = 8,
  ST_TIMEOUT = 16,
  ST_BAD_ARG = 32,
  ST_CAND_OVERFLOW = 64,  // fused records: more candidates than the list holds
  ST_INEXACT = 128        // fused records: a reduced value could not be certified
};

// Fused per-order records (nplet mode 3): ten thresholds per order slot, kept
// as order-preserving 32-bit keys.  Slot m (0..4) bounds measure m from
// above ("a nplet with a value at or below it is a candidate for the
// minimum"), slot 5 + m from below (candidates for the maximum); for the
// measure the top lists rank, slot m and 5 + m bound the smallest and the
// largest top lists instead.  A key of 0 means "no bound".
constexpr int FUSE_NTHR = 10;

// One block's partial reduction over one launch (one order).  Values are
// widened to double; ids are global ids.
struct PartRec {
  double vmin[5], vmax[5];
  unsigned long long imin[5], imax[5];
  double s_lr, s_sp, s_ls;  // sums of log det R_S, sum_j log p_j, sum_i log Sigma_ii
  unsigned long long count, neg, notpd;
  int top_hi, top_lo;       // valid entries in this block's top lists
};

struct TopEnt {
  double v;
  unsigned long long id;
};
static_assert(sizeof(TopEnt) == sizeof(thoi_top_entry), "layout");

// Constants of the combine step for one order k (Methods eqs. TC, DTC,
// O-info, S-info on the correlation matrix R = D^-1/2 Sigma D^-1/2):
//   TC  = -1/2 Lr + tc_c
//   DTC =  1/2 (Lr + Sp) + dtc_c
//   O = TC - DTC,  S = TC + DTC
//   H   = h_c + 1/2 (Lr + Ls)
// with Lr = log det R_S, Sp = sum_j log (R_S^-1)_jj, Ls = sum_{i in S} log Sigma_ii.
// The constants carry 1/2 k log(2 pi e) and the optional bias terms.
struct Combine {
  double h_c, tc_c, dtc_c;
  int top;  // measure the top-M lists rank (thoi_measure; O for the records API)
  int pad;
};

// Everything a nplet kernel needs for one order.
struct NpletArgs {
  int N;
  int k;
  const float* R32;     // N x N correlation, FP32 (row-major, stride N)
  const double* R64;    // N x N correlation, FP64
  const double* ls;     // log Sigma_ii, N entries
  const unsigned long long* binom;  // NB x NB table C(n, m)
  unsigned long long rank_begin, rank_end;  // lexicographic ranks within order k
  unsigned long long id_base;  // global id of rank 0 of this order
  Combine cmb;
  float tau_piv, tau_tr;
  // outputs
  int mode;             // 0: per-nplet SoA, 1: reduction partials
  void* out;            // mode 0: SoA base
  int out_f64;
  int out_sel;          // mode 0: 0 = the five measures (SoA); m + 1 = measure m alone (one row)
  unsigned long long out_n;      // stride between measures in `out`
  unsigned long long out_first;  // global id stored at out index 0
  PartRec* part;        // mode 1 and 3: [gridDim.x]
  TopEnt* part_top;     // mode 1: [gridDim.x][2][top_m]
  int top_m;
  // mode 3 (fused records): thresholds of this order slot (FUSE_NTHR keys),
  // and the candidate list the kernel appends to (ids; three FP32 arrays of
  // log det R_S, sum_j log p_j, sum_i log Sigma_ii at cand_b[m * cand_cap + e]).
  // The list is cut into cand_nseg segments of cand_seg entries; block b
  // appends to segment b % cand_nseg (counter cand_count[segment]), which
  // spreads the appends' atomics over several addresses.
  // mode 4 (sample bounds): the kernel evaluates sampled nplets and adds
  // their extremes to thr_keys (see launch_fused_sample).
  const unsigned* thr_keys;
  unsigned long long* cand_ids;
  float* cand_b;
  unsigned long long* cand_count;
  unsigned long long cand_cap;
  unsigned long long cand_seg;
  int cand_nseg;
  unsigned char* cand_ws;  // selection workspace of the candidate reduction (cand_ws_bytes())
  // FP64 re-factor list (FP32 kernels append; the re-factor kernel reads)
  unsigned long long* flag_ids;
  unsigned long long* flag_count;
  unsigned long long flag_cap;
  int* status;
  const int* cancel;    // device flag polled per round (may be null)
  // prefix-shared kernels: a zeroed device counter from which the warps take
  // their prefixes, 32 at a time (null: a static split over the grid)
  unsigned long long* work_counter;
};

// ------------------------------------------------------------------ launchers
// Maximum resident blocks per SM of a kernel at a dynamic shared-memory size,
// with the shared-memory attribute set; cached per (kernel, size) so that
// repeated launches do not pay for the occupancy query.
cudaError_t occupancy_cached(const void* fn, int block, size_t smem, int* occ);
struct Shape {
  int blocks_per_sm;  // 0 = occupancy maximum
  int chunk;          // nplets (prefixes for the prefix-shared kernel) per thread per round, 1..8
  int lanes;          // lanes per nplet: 1 (one-thread kernel), 2 or 4 (lane-group kernel)
  int prefix;         // prefix-shared kernels (whole orders, KPFX_MIN <= k <= KPFX_MAX):
                      // 1 shares a (k-1)-prefix, 2 a (k-2)-prefix, 3 a (k-2)-prefix with
                      // the last variables two at a time, 4 a (k-3)-prefix (from
                      // order 5) and 5 a (k-4)-prefix (from order 6), both with the
                      // last variables two at a time; 0 dense
};
constexpr int KPFX_MIN = 3;   // orders with a prefix-shared kernel
constexpr int KPFX_MAX = 20;   // the one-level kernel
constexpr int KPFX2_MAX = 24;  // the two-, three- and four-level kernels
// Built-in launch shape of the FP32 kernel for order k (used when no tuned
// shape is cached).
Shape default_shape(int k);
// Whether a (k, lanes) kernel instance exists.
bool shape_available(int k, int lanes);

// Workspace of the copula front end (device pointers owned by the context).
struct CopulaWs {
  int* rank;          // T x N
  double* ztab;       // T
  double* Z;          // N x T, variable-major
  double* mu;         // N
  double* sig64;      // N x N
  void* zh;           // Np x Tp BF16 (hi, mid, lo terms of Z - mu)
  void* zm;
  void* zl;
  double* part;       // n_chunks x Np x Np chunk tiles
  double* sig32acc;   // N x N, FP64 sum of the chunk tiles
};
struct CopulaWsSizes {
  int Np;
  long long Tp;
  int n_chunks;
};
void copula_ws_sizes(long long T, int N, CopulaWsSizes* z);
cudaError_t launch_copula(const void* X, int dtype, long long T, int N, long long ld,
                          const CopulaWs& w, int tc_cov, int* d_status, cudaStream_t s);
cudaError_t launch_normalise(const double* sig64, const double* sig32acc, int N, double* R64,
                             float* R32, double* ls, float* sig32_out, int* status,
                             cudaStream_t s);
cudaError_t launch_nplet_f32(const NpletArgs& a, const Shape& sh, int num_sms, cudaStream_t s,
                             int* grid_out, int max_blocks);
// Per-block reduction of n basis triples stored at basis[m * stride_elems + e]
// (element e has global id id0 + e); writes `grid` partials.
// seed_thr: device scratch for 2 floats (starting top-M thresholds), or null.
cudaError_t launch_reduce_basis(const float* basis, unsigned long long stride_elems,
                                unsigned long long n, unsigned long long id0, Combine cmb,
                                int top_m, float* seed_thr, PartRec* part, TopEnt* part_top,
                                int num_sms, int max_blocks, cudaStream_t s, int* grid_out);
cudaError_t launch_reduce_basis64(const double* basis, unsigned long long stride_elems,
                                  unsigned long long n, unsigned long long id0, Combine cmb,
                                  int top_m, PartRec* part, TopEnt* part_top, int num_sms,
                                  int max_blocks, cudaStream_t s, int* grid_out);
// Fused records of one order slot: the starting thresholds from a sample of
// the slot's nplets (FP32, every sampled nplet evaluated directly; keys added
// with atomicMax into thr_keys, which must be zero beforehand) ...
cudaError_t launch_fused_sample(const NpletArgs& a, int num_sms, cudaStream_t s);
int fused_sample_per_thread(unsigned long long n, int top_m);
size_t cand_ws_bytes();
int cand_partials(int nseg);  // partial records the candidate reduction writes
constexpr int FUSE_NSEG = 16;  // candidate-list segments (and candidate-reduction blocks)
// ... and, after the nplet launch, the reduction of the candidate list into
// per-block partials holding the extremes and top lists only; block 0 also
// carries the count of FP32 nplets (rank range minus the flagged ones).
cudaError_t launch_reduce_candidates(const NpletArgs& a, int num_sms, int max_blocks,
                                     PartRec* part, TopEnt* part_top, cudaStream_t s,
                                     int* grid_out);
cudaError_t launch_reduce_list64(const double* basis, unsigned long long stride_elems,
                                 const unsigned long long* ids, const unsigned long long* count,
                                 unsigned long long cap, Combine cmb, int top_m, PartRec* part,
                                 TopEnt* part_top, int num_sms, int max_blocks, cudaStream_t s,
                                 int* grid_out);
// Radix-select reductions (the candidate reduction's kernels on other
// sources): every field of the record from one streaming pass, the top-M
// lists from two histogram passes and one sort of the survivors.  More than
// SEL_SURV survivors (values tied within 2^-13 relative of the M-th) raise
// ST_INEXACT in *status: the request is then repeated with the streaming
// reductions.  ws: sel_ws_bytes() of device memory, one per stream in flight.
// A dense range of FP32 basis values (ids id0 + position; NaN = reduced from
// the re-factor list):
size_t sel_ws_bytes();
cudaError_t launch_select_basis(const float* basis, unsigned long long stride_elems,
                                unsigned long long n, unsigned long long id0, Combine cmb,
                                int top_m, unsigned char* ws, int* status, PartRec* part,
                                TopEnt* part_top, int max_blocks, cudaStream_t s, int* grid_out);
// A dense range of FP64 basis values (ids id0 + position; NaN = not
// positive definite):
cudaError_t launch_select_basis64(const double* basis, unsigned long long stride_elems,
                                  unsigned long long n, unsigned long long id0, Combine cmb,
                                  int top_m, unsigned char* ws, int* status, PartRec* part,
                                  TopEnt* part_top, int max_blocks, cudaStream_t s,
                                  int* grid_out);
// A re-factor list of FP64 basis values (count on the device, at most cap
// entries; NaN = not positive definite):
cudaError_t launch_select_list64(const double* basis, unsigned long long stride_elems,
                                 const unsigned long long* ids, const unsigned long long* count,
                                 unsigned long long cap, Combine cmb, int top_m,
                                 unsigned char* ws, int* status, PartRec* part, TopEnt* part_top,
                                 int max_blocks, cudaStream_t s, int* grid_out);
// FP64 kernels with shared-memory matrices: one thread per nplet (G = 1) or
// G lanes per nplet, 128 threads per block.
struct F64Cfg {
  int G;
  size_t smem;
};
F64Cfg f64_config(int N, int k);
// Nplets per block of the FP64 shared-memory kernel for (N, k) (never 0).
int f64s_threads(int N, int k, size_t* smem_out);
cudaError_t launch_nplet_f64s(const NpletArgs& a, bool list, double* b64,
                              unsigned long long bstride, int num_sms, cudaStream_t s,
                              int* grid_out, int max_blocks);
cudaError_t launch_nplet_f64(const NpletArgs& a, int num_sms, cudaStream_t s, int* grid_out,
                             int max_blocks);
cudaError_t launch_refactor(const NpletArgs& a, int num_sms, cudaStream_t s, int* grid_out,
                            int max_blocks);
// One order slot of a merge: where its FP32 and FP64 partials live.
struct MergeDesc {
  int p32_off, g32;   // first partial and count (FP32 path or FP64 path)
  int p64_off, g64;   // FP64 re-factor partials
  int k;
  int pad;
  Combine cmb;
  const unsigned long long* refactored;  // device counter of re-factored nplets (or null)
  // fused records: the slot's threshold keys (null otherwise); the merge
  // certifies the record against them and raises ST_INEXACT in *status
  const unsigned* thr_keys;
  int* status;
};
constexpr int MAX_SLOTS = 64;
struct MergeDescs {
  MergeDesc d[MAX_SLOTS];
};
// Batched merge: descriptors and per-slot output places in device memory;
// gmax = the largest g32 + g64 of any slot.
cudaError_t launch_merge_arr(const MergeDesc* D, int n_slots, int gmax, const PartRec* p32,
                             const TopEnt* t32, const PartRec* p64, const TopEnt* t64, int top_m,
                             thoi_order_record* const* recp, TopEnt* const* topp,
                             cudaStream_t s);
cudaError_t launch_merge(const MergeDescs& D, int n_slots, const PartRec* p32, const TopEnt* t32,
                         const PartRec* p64, const TopEnt* t64, int top_m, thoi_order_record* recs,
                         TopEnt* tops, cudaStream_t s);
cudaError_t launch_unrank_ids(int N, const int* d_orders, const unsigned long long* d_offsets,
                              int n_orders, const unsigned long long* binom,
                              const unsigned long long* ids, long long n, int kmax,
                              int8_t* idx_out, cudaStream_t s);
cudaError_t launch_grad_pass(const NpletArgs& a, double* Gpart, int grid, int measure, bool list,
                             cudaStream_t s);
cudaError_t launch_grad_finish(const double* Gpart, int nblk, const double* sig64, int N, float* out,
                               cudaStream_t s);

// Simulated annealing: n_chains independent chains (see anneal.cu).  D = 1
// evaluates the measure of one dataset (R0, ls0; a thread per chain, tables
// in shared memory); D > 1 a group objective (a warp per chain; Rs, lss:
// device arrays of D device pointers).  cmb_tab: D x (khi + 1) combine
// constants (row d, order k).
cudaError_t launch_anneal(const double* const* Rs, const double* const* lss, int D,
                          int objective, int N, int klo, int khi, const Combine* cmb_tab,
                          const double* R0, const double* ls0, int n_chains, int iters, double T0,
                          double alpha, int patience, int measure, int maximize,
                          unsigned long long seed,
                          unsigned long long* final_mask, double* final_val,
                          unsigned long long* best_mask, double* best_val,
                          unsigned long long* accepted, cudaStream_t s);
// Group objectives: fold one dataset's status and re-factor count; combine the
// D x ld value matrix into the objective (per-nplet `out` and/or an FP64
// basis with stride bstride; count: optional device list length); copy the
// objective's statistics into every measure slot of the records.
cudaError_t launch_group_fold(const int* status, const unsigned long long* flag_count,
                              unsigned long long flag_cap, int* gstatus, unsigned long long* gnref,
                              cudaStream_t s);
cudaError_t launch_group_combine(const double* V, unsigned long long ld, unsigned long long n,
                                 const unsigned long long* count, int D, int objective,
                                 double* out, double* basis, unsigned long long bstride,
                                 int num_sms, cudaStream_t s);
cudaError_t launch_group_fix(thoi_order_record* recs, int n, cudaStream_t s);
// Greedy expansion on the device: parents = the first min(top_count, kappa)
// entries of `tops` (one side of the previous order's records, order kp);
// distinct candidates of order kp + 1 appended as lexicographic ranks to ids
// (count: device counter, zeroed by the caller; table: tsize zeroed slots,
// tsize a power of two >= 2 kappa N).
cudaError_t launch_greedy_expand(const thoi_order_record* rec, const TopEnt* tops, int kappa,
                                 int N, int kp, const unsigned long long* binom,
                                 unsigned long long* table, unsigned long long tsize,
                                 unsigned long long* ids, unsigned long long* count,
                                 cudaStream_t s);

// ------------------------------------------------------------------ multi-dataset batch
// Many datasets of uneven (N, T) in one graph: per order k one persistent
// nplet launch walks a list of tiles (dataset, rank range) of every dataset,
// one reduction launch walks a list of reduction tiles, then one FP64
// re-factor launch and one list-reduction launch cover every dataset's
// flagged nplets (grid.y = slot), and one merge launch writes every record.
struct BatchDataset {
  const float* R32;   // N x N correlation, FP32
  const double* R64;  // N x N correlation, FP64
  const double* ls;   // log Sigma_ii
  int N;
  float tau_piv, tau_tr;
  int pad;
};
// One (dataset, order) pair with at least one nplet.
struct BatchSlot {
  int d, k;
  unsigned long long n;        // C(N_d, k)
  unsigned long long id_base;  // global id of rank 0 within dataset d's enumeration
  unsigned long long flag_off, flag_cap;  // region of the flag list (and FP64 basis)
  Combine cmb;
};
// Tile of the persistent batched kernel: ranks [r0, r0 + n) of a slot
// (n <= 2^16, order k), reduced into partial record pidx.
struct BatchFTile {
  unsigned long long r0;
  unsigned n;
  int slot;
  int pidx;
  int k;
};
struct BatchFArgs {
  const BatchDataset* ds;
  const BatchSlot* slots;
  const BatchFTile* tiles;
  int n_tiles;
  int top_m;
  const unsigned long long* binom;  // NB x NB
  unsigned long long* flag_ids;
  unsigned long long* flag_counts;  // one counter per slot
  PartRec* part;
  TopEnt* part_top;
  unsigned* tile_counter;           // zero before the launch
  // per slot, the tightest top-M bounds any of its tiles has found (two
  // order-preserving keys, the smallest side complemented; zero before the
  // launch = none): later tiles of the slot start from them.  Null: none.
  unsigned* slot_thr;
  int* status;
  const int* cancel;
  int chunk_k[KBATCH_MAX + 1];      // nplets per thread per round, by order
};
// Orders of each band of the persistent batched kernel (one kernel per band).
constexpr int BATCH_BANDS = 4;
constexpr int BATCH_BAND_LO[BATCH_BANDS] = {1, 9, 15, 18};
constexpr int BATCH_BAND_HI[BATCH_BANDS] = {8, 14, 17, 20};
// One launch of band `band` over the tiles in b (all of the band's orders);
// blocks_per_sm 0 = the occupancy maximum.
cudaError_t launch_batch_fused(int band, bool wide, const BatchFArgs& b, int maxN,
                               int blocks_per_sm, int num_sms, cudaStream_t s, int* grid_out);
// FP64 re-factor of the flagged nplets of slots [slot0, slot0 + n_slots),
// grid (bx, n_slots); basis values at b64[m * lstride + flag_off + e].
cudaError_t launch_refactor_batch(const BatchDataset* ds, const BatchSlot* slots, int slot0,
                                  int n_slots, int maxN, int k, bool wide,
                                  const unsigned long long* binom,
                                  const unsigned long long* flag_ids,
                                  unsigned long long* flag_counts, double* b64,
                                  unsigned long long lstride, int* status, int bx,
                                  cudaStream_t s);
// Reduction of those lists: partial (slot, x) at part[(slot) * bx + x].
cudaError_t launch_reduce_list_batch(const double* b64, unsigned long long lstride,
                                     const BatchSlot* slots, int slot0, int n_slots,
                                     const unsigned long long* flag_ids,
                                     const unsigned long long* flag_counts, int top_m,
                                     PartRec* part, TopEnt* part_top, int bx, cudaStream_t s);
// Group searches over D datasets sharing one candidate list: replicate the
// list into D regions of stride cap_pad with per-slot counters (for the
// batched FP64 kernel), and pick one measure per dataset from the batched
// basis into the D x cap_pad value matrix.
cudaError_t launch_group_replicate(const unsigned long long* ids, const unsigned long long* count,
                                   unsigned long long cap, int D, unsigned long long cap_pad,
                                   unsigned long long* ids_rep, unsigned long long* counts_rep,
                                   cudaStream_t s);
cudaError_t launch_group_pick_batch(const double* b64, unsigned long long lstride,
                                    unsigned long long cap_pad, int D, const BatchSlot* slots,
                                    const unsigned long long* count, unsigned long long cap,
                                    int measure, double* V, cudaStream_t s);

// ------------------------------------------------------------------ device helpers
#ifdef __CUDACC__

__device__ __forceinline__ unsigned long long binom_at(const unsigned long long* b, int n, int m) {
  return b[n * NB + m];
}

// Lexicographic rank r of a k-subset of {0..N-1} -> reversed bitmask (bit
// N-1-c set for every member c).  Combinatorial number system: with
// r' = C(N,k) - 1 - r, the members satisfy r' = sum_i C(d_i, k-i) with
// d_i = N-1-c_i strictly decreasing; each d_i is the largest d whose
// binomial still fits into what is left of r'.
template <typename M>
__device__ __forceinline__ M unrank_mask(unsigned long long r, int k, int N,
                                         const unsigned long long* b) {
  unsigned long long rr = binom_at(b, N, k) - 1ull - r;
  M mask = 0;
  int d = N - 1;
  for (int i = 0; i < k; i++) {
    const int m = k - i;
    unsigned long long cd = binom_at(b, d, m);
    while (cd > rr) {
      d--;
      cd = binom_at(b, d, m);
    }
    rr -= cd;
    mask |= (M)1 << d;
    d--;
  }
  return mask;
}

__device__ __forceinline__ int ctz_m(unsigned int x) { return __ffs(x) - 1; }
__device__ __forceinline__ int ctz_m(unsigned long long x) { return __ffsll((long long)x) - 1; }
__device__ __forceinline__ int hibit(unsigned int x) { return 31 - __clz(x); }
__device__ __forceinline__ int hibit(unsigned long long x) { return 63 - __clzll((long long)x); }

// Lexicographic successor in the reversed-bitmask encoding: lexicographic
// order of sorted tuples is decreasing numeric order of the reversed mask,
// so the successor is the next smaller N-bit number with the same number of
// ones, i.e. the complement of the next larger number with the complement's
// popcount (Gosper's rule).
template <typename M>
__device__ __forceinline__ M lex_succ(M x, M full) {
  M y = ~x & full;
  M t = y & (~y + 1);
  M r = y + t;
  M nx = r | (((y ^ r) >> 2) >> ctz_m(t));
  return ~nx & full;
}

#endif  // __CUDACC__

}  // namespace thoi
