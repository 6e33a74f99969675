/*
 * FP64 CPU oracle for exhaustive Gaussian-copula higher-order information.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg may load this library.  The product path (the CUDA
 * library) never calls it, links it or shares code with it.
 *
 * Every function restates a definition of the paper (arXiv 2501.03381) in the
 * most literal form, with no blocking, fusion or algebraic shortcut:
 *   - rank / copula / covariance : Supplementary Methods, eq.
 *     "gaussian_copula_covariance_estimator" (rank -> /(T+1) -> inverse
 *     normal CDF -> covariance operator).
 *   - entropy                    : Supplementary Methods, eq.
 *     "gaussian_differential_entropy", H = 1/2 log((2 pi e)^n |Sigma|),
 *     with |Sigma| from an LU factorisation with partial pivoting.
 *   - TC, DTC, O, S              : Methods, eqs. "TC", "DTC", "O-info",
 *     "S-info", each evaluated from entropies exactly as written (the
 *     conditional entropy H(X_j | X_-j) = H(X) - H(X_-j)); every
 *     leave-one-out entropy gets its own LU.
 *   - enumeration                : Supplementary Methods, eq. "comb"
 *     (all k-subsets of N), in lexicographic order of the sorted index tuple.
 *   - bias corrector             : Supplementary Methods, eq.
 *     "bias_corrector", read with the factor 1/2 on the digamma sum (the
 *     Wishart expectation of log det); off unless T_bias > 0.
 *
 * Readings where the paper is silent (the same list is kept with the design
 * notes): ordinal 0-based ranks with ties broken by sample index, made
 * 1-based for u = (r+1)/(T+1); the covariance is centred and divided by
 * T-1; nplets whose determinant is <= 0 are marked not positive definite
 * and get NaN measures.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_NONFINITE 2
#define ORC_ERR_SELFCHECK 3
#define ORC_ERR_NOMEM 4
#define ORC_MAXN 64

static const double LOG_2PIE = 2.8378770664093454835606594728112; /* log(2 pi e) */

/* ------------------------------------------------------------------------ */
/* Binomial coefficients by Pascal's triangle (exact in uint64 for n <= 64). */
static uint64_t g_binom[ORC_MAXN + 1][ORC_MAXN + 1];
static int g_binom_ready = 0;

static void binom_init(void) {
  if (g_binom_ready) return;
  for (int n = 0; n <= ORC_MAXN; n++) {
    g_binom[n][0] = 1;
    for (int k = 1; k <= ORC_MAXN; k++)
      g_binom[n][k] = (n == 0) ? 0 : g_binom[n - 1][k - 1] + g_binom[n - 1][k];
  }
  g_binom_ready = 1;
}

uint64_t orc_binom(int n, int k) {
  binom_init();
  if (n < 0 || k < 0 || n > ORC_MAXN || k > ORC_MAXN) return 0;
  return g_binom[n][k];
}

/* Number of nplets over the listed orders (Supp. eq. "comb"). */
uint64_t orc_count(int N, const int32_t* orders, int n_orders) {
  uint64_t s = 0;
  for (int o = 0; o < n_orders; o++) s += orc_binom(N, orders[o]);
  return s;
}

/* ------------------------------------------------------------------------ */
/* Rank: stable sort of (value, sample index) per column.  The 0-based
 * position in the sorted order is the ordinal rank; equal values keep
 * sample order.  -0.0 and +0.0 compare equal.  NaN/Inf is an error.       */
typedef struct { double v; int64_t i; } orc_pair;

static int cmp_pair(const void* a, const void* b) {
  const orc_pair* x = (const orc_pair*)a;
  const orc_pair* y = (const orc_pair*)b;
  if (x->v < y->v) return -1;
  if (x->v > y->v) return 1;
  return (x->i < y->i) ? -1 : (x->i > y->i) ? 1 : 0;
}

int orc_rank(const double* X, int64_t T, int64_t N, int64_t ld, int32_t* R) {
  if (!X || !R || T < 1 || N < 1 || ld < N) return ORC_ERR_ARG;
  for (int64_t t = 0; t < T; t++)
    for (int64_t j = 0; j < N; j++)
      if (!isfinite(X[t * ld + j])) return ORC_ERR_NONFINITE;
  orc_pair* p = (orc_pair*)malloc(sizeof(orc_pair) * (size_t)T);
  if (!p) return ORC_ERR_NOMEM;
  for (int64_t j = 0; j < N; j++) {
    for (int64_t t = 0; t < T; t++) { p[t].v = X[t * ld + j]; p[t].i = t; }
    qsort(p, (size_t)T, sizeof(orc_pair), cmp_pair);
    for (int64_t r = 0; r < T; r++) R[p[r].i * N + j] = (int32_t)r;
  }
  free(p);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Inverse standard normal CDF.  Independent method: bisection on the
 * lower-tail CDF Phi(z) = erfc(-z/sqrt 2)/2 until the bracket stops
 * shrinking, then Newton polishing with phi(z).  For a probability above 1/2
 * the symmetric lower-tail problem is solved and negated, so the tail value
 * keeps full relative precision.                                          */
static double Phi_lower(double z) { return 0.5 * erfc(-z / 1.4142135623730950488); }

static double ndtri_lower(double p) { /* 0 < p <= 1/2, result <= 0 */
  double lo = -40.0, hi = 0.0;
  for (int it = 0; it < 200; it++) {
    double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    if (Phi_lower(mid) < p) lo = mid; else hi = mid;
  }
  double z = (fabs(Phi_lower(lo) - p) <= fabs(Phi_lower(hi) - p)) ? lo : hi;
  for (int it = 0; it < 3; it++) {
    double f = Phi_lower(z) - p;
    double d = exp(-0.5 * z * z) * 0.39894228040143267794;
    if (d <= 0) break;
    double zn = z - f / d;
    if (!(fabs(Phi_lower(zn) - p) < fabs(f))) break;
    z = zn;
  }
  return z;
}

/* Phi^{-1}(num/den) for 0 < num < den, evaluated from the nearer tail. */
double orc_ndtri_ratio(double num, double den) {
  if (!(num > 0 && num < den)) return NAN;
  if (2.0 * num == den) return 0.0;
  if (2.0 * num < den) return ndtri_lower(num / den);
  return -ndtri_lower((den - num) / den);
}

double orc_ndtri(double u) {
  if (!(u > 0 && u < 1)) return NAN;
  if (u == 0.5) return 0.0;
  if (u < 0.5) return ndtri_lower(u);
  return -ndtri_lower(1.0 - u);
}

/* Copula transform and covariance (Supp. eq.
 * gaussian_copula_covariance_estimator): u = (r+1)/(T+1), z = Phi^{-1}(u),
 * mu_j = mean_t z_tj, Sigma_ij = sum_t (z_ti-mu_i)(z_tj-mu_j)/(T-1).
 * Z (T x N, may be NULL) receives the transformed samples.                */
int orc_copula_cov(const double* X, int64_t T, int64_t N, int64_t ld, double* Z,
                   double* Sigma) {
  if (!X || !Sigma || T < 2 || N < 1 || ld < N) return ORC_ERR_ARG;
  int32_t* R = (int32_t*)malloc(sizeof(int32_t) * (size_t)(T * N));
  double* Zl = (double*)malloc(sizeof(double) * (size_t)(T * N));
  double* mu = (double*)malloc(sizeof(double) * (size_t)N);
  if (!R || !Zl || !mu) { free(R); free(Zl); free(mu); return ORC_ERR_NOMEM; }
  int st = orc_rank(X, T, N, ld, R);
  if (st) { free(R); free(Zl); free(mu); return st; }
  for (int64_t t = 0; t < T; t++)
    for (int64_t j = 0; j < N; j++)
      Zl[t * N + j] = orc_ndtri_ratio((double)R[t * N + j] + 1.0, (double)T + 1.0);
  for (int64_t j = 0; j < N; j++) {
    long double s = 0;
    for (int64_t t = 0; t < T; t++) s += Zl[t * N + j];
    mu[j] = (double)(s / (long double)T);
  }
  for (int64_t i = 0; i < N; i++)
    for (int64_t j = 0; j <= i; j++) {
      long double s = 0;
      for (int64_t t = 0; t < T; t++)
        s += ((long double)Zl[t * N + i] - mu[i]) * ((long double)Zl[t * N + j] - mu[j]);
      double v = (double)(s / (long double)(T - 1));
      Sigma[i * N + j] = v;
      Sigma[j * N + i] = v;
    }
  if (Z) memcpy(Z, Zl, sizeof(double) * (size_t)(T * N));
  free(R); free(Zl); free(mu);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Enumeration.  Within an order, k-subsets in lexicographic order of the
 * sorted tuple c_0 < ... < c_{k-1}; orders follow the caller's list; the
 * global id is the running counter over that sequence.                    */

/* Lexicographic successor: bump the rightmost c_i that can still grow and
 * reset the tail.  Returns 0 after the last subset.                        */
static int lex_next(int* c, int k, int N) {
  int i = k - 1;
  while (i >= 0 && c[i] == N - k + i) i--;
  if (i < 0) return 0;
  c[i]++;
  for (int j = i + 1; j < k; j++) c[j] = c[j - 1] + 1;
  return 1;
}

/* Lexicographic unrank by counting completions: the number of k-subsets
 * whose i-th element is x given the prefix is C(N-1-x, k-1-i).             */
static void lex_unrank(uint64_t r, int k, int N, int* c) {
  int prev = -1;
  for (int i = 0; i < k; i++) {
    int x = prev + 1;
    for (;;) {
      uint64_t cnt = orc_binom(N - 1 - x, k - 1 - i);
      if (r < cnt) break;
      r -= cnt;
      x++;
    }
    c[i] = x;
    prev = x;
  }
}

/* Split a global id into (order slot, rank within the order). */
static int split_id(int N, const int32_t* orders, int n_orders, uint64_t id,
                    int* slot, uint64_t* rank) {
  for (int o = 0; o < n_orders; o++) {
    uint64_t c = orc_binom(N, orders[o]);
    if (id < c) { *slot = o; *rank = id; return 1; }
    id -= c;
  }
  return 0;
}

/* Walk the ids [id_begin, id_end) by successor and write each subset
 * (k indices, padded with -1 to kmax) -- used to pin the enumeration.      */
int orc_enumerate(int N, const int32_t* orders, int n_orders, uint64_t id_begin,
                  uint64_t id_end, int kmax, int8_t* idx_out) {
  if (N < 1 || N > ORC_MAXN || id_end < id_begin) return ORC_ERR_ARG;
  for (int o = 0; o < n_orders; o++)
    if (orders[o] < 1 || orders[o] > N || orders[o] > kmax) return ORC_ERR_ARG;
  if (id_end > orc_count(N, orders, n_orders)) return ORC_ERR_ARG;
  if (id_end == id_begin) return ORC_OK;
  int slot; uint64_t r;
  split_id(N, orders, n_orders, id_begin, &slot, &r);
  int c[ORC_MAXN];
  int k = orders[slot];
  lex_unrank(r, k, N, c);
  for (uint64_t id = id_begin; id < id_end; id++) {
    int8_t* row = idx_out + (size_t)(id - id_begin) * (size_t)kmax;
    for (int i = 0; i < kmax; i++) row[i] = (i < k) ? (int8_t)c[i] : (int8_t)-1;
    if (!lex_next(c, k, N)) {
      slot++;
      if (slot >= n_orders) break;
      k = orders[slot];
      for (int i = 0; i < k; i++) c[i] = i;
    }
  }
  return ORC_OK;
}

/* Unrank each listed id independently (counting method). */
int orc_unrank_ids(int N, const int32_t* orders, int n_orders, const uint64_t* ids,
                   int64_t n, int kmax, int8_t* idx_out) {
  for (int64_t q = 0; q < n; q++) {
    int slot; uint64_t r;
    if (!split_id(N, orders, n_orders, ids[q], &slot, &r)) return ORC_ERR_ARG;
    int c[ORC_MAXN];
    int k = orders[slot];
    if (k > kmax) return ORC_ERR_ARG;
    lex_unrank(r, k, N, c);
    int8_t* row = idx_out + (size_t)q * (size_t)kmax;
    for (int i = 0; i < kmax; i++) row[i] = (i < k) ? (int8_t)c[i] : (int8_t)-1;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* log|det A| by LU with partial pivoting (A is n x n row-major, destroyed).
 * Returns the sign of det A (+1, -1) or 0 when a pivot is exactly zero.   */
static int lu_logdet(double* A, int n, double* logdet) {
  int sign = 1;
  double ld = 0.0;
  for (int p = 0; p < n; p++) {
    int piv = p;
    double best = fabs(A[p * n + p]);
    for (int i = p + 1; i < n; i++)
      if (fabs(A[i * n + p]) > best) { best = fabs(A[i * n + p]); piv = i; }
    if (best == 0.0 || !isfinite(best)) { *logdet = -INFINITY; return 0; }
    if (piv != p) {
      for (int j = 0; j < n; j++) {
        double t = A[p * n + j]; A[p * n + j] = A[piv * n + j]; A[piv * n + j] = t;
      }
      sign = -sign;
    }
    double d = A[p * n + p];
    if (d < 0) sign = -sign;
    ld += log(fabs(d));
    for (int i = p + 1; i < n; i++) {
      double f = A[i * n + p] / d;
      if (f == 0.0) continue;
      for (int j = p + 1; j < n; j++) A[i * n + j] -= f * A[p * n + j];
    }
  }
  *logdet = ld;
  return sign;
}

/* Digamma for x > 0: recurrence up to x >= 10, then the asymptotic series
 * psi(x) ~ ln x - 1/(2x) - sum_n B_2n / (2n x^{2n}).                        */
double orc_digamma(double x) {
  double r = 0.0;
  while (x < 10.0) { r -= 1.0 / x; x += 1.0; }
  double f = 1.0 / (x * x);
  double t = f * (-1.0 / 12 + f * (1.0 / 120 + f * (-1.0 / 252 + f * (1.0 / 240 +
             f * (-1.0 / 132 + f * (691.0 / 32760 + f * (-1.0 / 12)))))));
  return r + log(x) - 0.5 / x + t;
}

/* Bias of the Gaussian entropy of m variables from T samples (Supp. eq.
 * bias_corrector, with 1/2 on the digamma sum):
 * eta_m = 1/2 [ m log(2/(T-1)) + sum_{j=1..m} psi((T-j)/2) ].             */
double orc_bias_eta(int m, int64_t T) {
  if (m <= 0) return 0.0;
  double s = (double)m * log(2.0 / (double)(T - 1));
  for (int j = 1; j <= m; j++) s += orc_digamma(0.5 * (double)(T - j));
  return 0.5 * s;
}

/* Entropy of the sub-vector idx[0..n) (eq. gaussian_differential_entropy),
 * minus the bias eta_n when T_bias > 0.  Returns 0 when det <= 0.         */
static int entropy_of(const double* Sigma, int N, const int* idx, int n, int64_t T_bias,
                      double* H) {
  if (n == 0) { *H = 0.0; return 1; }
  double A[ORC_MAXN * ORC_MAXN];
  for (int a = 0; a < n; a++)
    for (int b = 0; b < n; b++) A[a * n + b] = Sigma[idx[a] * N + idx[b]];
  double ld;
  int s = lu_logdet(A, n, &ld);
  if (s <= 0) { *H = NAN; return 0; }
  double h = 0.5 * ((double)n * LOG_2PIE + ld);
  if (T_bias > 0) h -= orc_bias_eta(n, T_bias);
  *H = h;
  return 1;
}

/* The five measures of one nplet, each from its definition.  Returns 1 when
 * every entropy exists, 0 when some subset is not positive definite (all
 * five set to NaN), -1 when the two forms of eq. O-info disagree.          */
static int measures_one(const double* Sigma, int N, const int* c, int k, int64_t T_bias,
                        double out[5]) {
  double HS, Hj[ORC_MAXN], Hm[ORC_MAXN];
  int sub[ORC_MAXN];
  int ok = entropy_of(Sigma, N, c, k, T_bias, &HS);
  for (int j = 0; j < k && ok; j++) {
    ok &= entropy_of(Sigma, N, &c[j], 1, T_bias, &Hj[j]);
    int q = 0;
    for (int i = 0; i < k; i++) if (i != j) sub[q++] = c[i];
    ok &= entropy_of(Sigma, N, sub, k - 1, T_bias, &Hm[j]);
  }
  if (!ok) { for (int m = 0; m < 5; m++) out[m] = NAN; return 0; }
  /* eq. TC: sum_j H(X_j) - H(X^n) */
  long double tc = -(long double)HS;
  for (int j = 0; j < k; j++) tc += Hj[j];
  /* eq. DTC: H(X^n) - sum_j H(X_j | X_-j), H(X_j|X_-j) = H(X^n) - H(X_-j) */
  long double dtc = HS;
  for (int j = 0; j < k; j++) dtc -= ((long double)HS - Hm[j]);
  /* eq. O-info (first form) and eq. S-info */
  long double o = tc - dtc, s = tc + dtc;
  /* eq. O-info (second form) as a self check */
  long double o2 = (long double)(k - 2) * HS;
  for (int j = 0; j < k; j++) o2 += (long double)Hj[j] - Hm[j];
  out[0] = HS; out[1] = (double)tc; out[2] = (double)dtc; out[3] = (double)o; out[4] = (double)s;
  if (fabsl(o - o2) > 1e-8L * (1.0L + fabsl(o))) return -1;
  return 1;
}

/* Measures of every nplet with id in [id_begin, id_end).  out is SoA:
 * out[m * n + (id - id_begin)] for m = H, TC, DTC, O, S.  flags[i] = 1 when
 * the nplet is not positive definite.  Returns ORC_ERR_SELFCHECK if the two
 * forms of O disagree anywhere.                                            */
int orc_measures(const double* Sigma, int N, const int32_t* orders, int n_orders,
                 uint64_t id_begin, uint64_t id_end, int64_t T_bias, double* out,
                 uint8_t* flags, int nthreads) {
  if (!Sigma || N < 1 || N > ORC_MAXN || id_end < id_begin) return ORC_ERR_ARG;
  for (int o = 0; o < n_orders; o++) if (orders[o] < 1 || orders[o] > N) return ORC_ERR_ARG;
  if (id_end > orc_count(N, orders, n_orders)) return ORC_ERR_ARG;
  binom_init();
  const uint64_t n = id_end - id_begin;
  const uint64_t CH = 2048;
  const int64_t nch = (int64_t)((n + CH - 1) / CH);
  int bad = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(|: bad)
#endif
  for (int64_t ch = 0; ch < nch; ch++) {
    uint64_t a = id_begin + (uint64_t)ch * CH;
    uint64_t b = a + CH < id_end ? a + CH : id_end;
    int slot; uint64_t r;
    split_id(N, orders, n_orders, a, &slot, &r);
    int c[ORC_MAXN];
    int k = orders[slot];
    lex_unrank(r, k, N, c);
    for (uint64_t id = a; id < b; id++) {
      double v[5];
      int st = measures_one(Sigma, N, c, k, T_bias, v);
      uint64_t i = id - id_begin;
      for (int m = 0; m < 5; m++) out[m * n + i] = v[m];
      if (flags) flags[i] = (st == 0) ? 1 : 0;
      if (st < 0) bad = 1;
      if (id + 1 < b && !lex_next(c, k, N)) {
        slot++;
        k = orders[slot];
        for (int q = 0; q < k; q++) c[q] = q;
      }
    }
  }
  return bad ? ORC_ERR_SELFCHECK : ORC_OK;
}

/* Measures of each listed id (independent unranking per id). */
int orc_measures_ids(const double* Sigma, int N, const int32_t* orders, int n_orders,
                     const uint64_t* ids, int64_t n, int64_t T_bias, double* out,
                     uint8_t* flags, int nthreads) {
  if (!Sigma || N < 1 || N > ORC_MAXN) return ORC_ERR_ARG;
  binom_init();
  int bad = 0, badid = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64) reduction(|: bad, badid)
#endif
  for (int64_t q = 0; q < n; q++) {
    int slot; uint64_t r;
    if (!split_id(N, orders, n_orders, ids[q], &slot, &r)) { badid = 1; continue; }
    int c[ORC_MAXN];
    int k = orders[slot];
    lex_unrank(r, k, N, c);
    double v[5];
    int st = measures_one(Sigma, N, c, k, T_bias, v);
    for (int m = 0; m < 5; m++) out[m * n + q] = v[m];
    if (flags) flags[q] = (st == 0) ? 1 : 0;
    if (st < 0) bad = 1;
  }
  if (badid) return ORC_ERR_ARG;
  return bad ? ORC_ERR_SELFCHECK : ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Gradient of L = sum over nplets of one measure with respect to Sigma,
 * entries treated as independent (the convention of d logdet / d Sigma =
 * Sigma^{-1}).  Per nplet, with P = Sigma_S^{-1} (explicit inverse by
 * Gauss-Jordan elimination with partial pivoting) and p_j = P_jj:
 *   d H / d Sigma_S   = 1/2 P
 *   d TC / d Sigma_S  = 1/2 [diag(1/Sigma_ii) - P]
 *   d DTC / d Sigma_S = 1/2 [P - P diag(1/p) P]
 *   d O / d Sigma_S   = 1/2 [diag(1/Sigma_ii) - 2P + P diag(1/p) P]
 *   d S / d Sigma_S   = 1/2 [diag(1/Sigma_ii) - P diag(1/p) P]
 * (from eq. gaussian_differential_entropy and d(Sigma^{-1})_jj =
 * -(P dSigma P)_jj).  The bias terms are constants and drop out.           */
static int invert_gj(const double* A0, int n, double* Ainv) {
  double A[ORC_MAXN * ORC_MAXN];
  memcpy(A, A0, sizeof(double) * (size_t)(n * n));
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) Ainv[i * n + j] = (i == j) ? 1.0 : 0.0;
  for (int p = 0; p < n; p++) {
    int piv = p;
    for (int i = p + 1; i < n; i++) if (fabs(A[i * n + p]) > fabs(A[piv * n + p])) piv = i;
    if (A[piv * n + p] == 0.0) return 0;
    if (piv != p)
      for (int j = 0; j < n; j++) {
        double t = A[p * n + j]; A[p * n + j] = A[piv * n + j]; A[piv * n + j] = t;
        t = Ainv[p * n + j]; Ainv[p * n + j] = Ainv[piv * n + j]; Ainv[piv * n + j] = t;
      }
    double d = A[p * n + p];
    for (int j = 0; j < n; j++) { A[p * n + j] /= d; Ainv[p * n + j] /= d; }
    for (int i = 0; i < n; i++) {
      if (i == p) continue;
      double f = A[i * n + p];
      if (f == 0.0) continue;
      for (int j = 0; j < n; j++) { A[i * n + j] -= f * A[p * n + j]; Ainv[i * n + j] -= f * Ainv[p * n + j]; }
    }
  }
  return 1;
}

/* measure: 0=H 1=TC 2=DTC 3=O 4=S.  G is N x N (row-major). */
int orc_grad(const double* Sigma, int N, const int32_t* orders, int n_orders, int measure,
             double* G, int nthreads) {
  if (!Sigma || !G || N < 1 || N > ORC_MAXN || measure < 0 || measure > 4) return ORC_ERR_ARG;
  binom_init();
  const uint64_t total = orc_count(N, orders, n_orders);
  const uint64_t CH = 4096;
  const int64_t nch = (int64_t)((total + CH - 1) / CH);
  int nt = 1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
  nt = omp_get_max_threads();
#endif
  long double* acc = (long double*)calloc((size_t)nt * (size_t)(N * N), sizeof(long double));
  if (!acc) return ORC_ERR_NOMEM;
  int bad = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static, 1) reduction(|: bad)
#endif
  for (int64_t ch = 0; ch < nch; ch++) {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    long double* Gt = acc + (size_t)tid * (size_t)(N * N);
    uint64_t a = (uint64_t)ch * CH;
    uint64_t b = a + CH < total ? a + CH : total;
    int slot; uint64_t r;
    split_id(N, orders, n_orders, a, &slot, &r);
    int c[ORC_MAXN];
    int k = orders[slot];
    lex_unrank(r, k, N, c);
    double S[ORC_MAXN * ORC_MAXN], P[ORC_MAXN * ORC_MAXN];
    for (uint64_t id = a; id < b; id++) {
      for (int x = 0; x < k; x++)
        for (int y = 0; y < k; y++) S[x * k + y] = Sigma[c[x] * N + c[y]];
      if (!invert_gj(S, k, P)) { bad = 1; }
      else {
        for (int x = 0; x < k; x++)
          for (int y = 0; y < k; y++) {
            long double pdp = 0;
            for (int j = 0; j < k; j++) pdp += (long double)P[x * k + j] * P[j * k + y] / P[j * k + j];
            long double dg = (x == y) ? 1.0L / Sigma[c[x] * N + c[x]] : 0.0L;
            long double g;
            switch (measure) {
              case 0: g = 0.5L * P[x * k + y]; break;
              case 1: g = 0.5L * (dg - P[x * k + y]); break;
              case 2: g = 0.5L * (P[x * k + y] - pdp); break;
              case 3: g = 0.5L * (dg - 2.0L * P[x * k + y] + pdp); break;
              default: g = 0.5L * (dg - pdp); break;
            }
            Gt[c[x] * N + c[y]] += g;
          }
      }
      if (id + 1 < b && !lex_next(c, k, N)) {
        slot++;
        k = orders[slot];
        for (int q = 0; q < k; q++) c[q] = q;
      }
    }
  }
  for (int i = 0; i < N * N; i++) {
    long double s = 0;
    for (int t = 0; t < nt; t++) s += acc[(size_t)t * (size_t)(N * N) + i];
    G[i] = (double)s;
  }
  free(acc);
  return bad ? ORC_ERR_SELFCHECK : ORC_OK;
}

/* Sum of one measure over the nplets of the listed orders that contain both
 * variables i and j (i == j: those containing i).  Only these nplets depend
 * on Sigma_ij, so a finite difference of this sum equals the finite
 * difference of the full objective.  Each nplet uses the literal
 * entropy-based measures (LU determinants), not the inverse.               */
int orc_objective_containing(const double* Sigma, int N, const int32_t* orders, int n_orders,
                             int measure, int i, int j, double* out, int nthreads) {
  if (!Sigma || !out || N < 1 || N > ORC_MAXN || i < 0 || j < 0 || i >= N || j >= N ||
      measure < 0 || measure > 4) return ORC_ERR_ARG;
  binom_init();
  int fixed[2] = {i < j ? i : j, i < j ? j : i};
  int nf = (i == j) ? 1 : 2;
  int others[ORC_MAXN], no = 0;
  for (int v = 0; v < N; v++) if (v != fixed[0] && v != fixed[nf - 1]) others[no++] = v;
  long double total = 0;
  int bad = 0;
  for (int o = 0; o < n_orders; o++) {
    int k = orders[o];
    int m = k - nf;
    if (m < 0 || m > no) continue;
    uint64_t cnt = orc_binom(no, m);
    const uint64_t CH = 1024;
    int64_t nch = (int64_t)((cnt + CH - 1) / CH);
    long double part = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static, 1) reduction(+: part) reduction(|: bad)
#endif
    for (int64_t ch = 0; ch < nch; ch++) {
      uint64_t a = (uint64_t)ch * CH, b = a + CH < cnt ? a + CH : cnt;
      int d[ORC_MAXN];
      if (m > 0) lex_unrank(a, m, no, d);
      for (uint64_t q = a; q < b; q++) {
        int c[ORC_MAXN], nc = 0, u = 0, f = 0;
        /* merge the sorted "others" picks with the fixed variables */
        while (u < m || f < nf) {
          int x = (u < m) ? others[d[u]] : 1 << 30;
          int y = (f < nf) ? fixed[f] : 1 << 30;
          if (x < y) { c[nc++] = x; u++; } else { c[nc++] = y; f++; }
        }
        double v[5];
        int st = measures_one(Sigma, N, c, k, 0, v);
        if (st <= 0) bad = 1;
        part += v[measure];
        if (m > 0 && q + 1 < b) lex_next(d, m, no);
      }
    }
    total += part;
  }
  *out = (double)total;
  return bad ? ORC_ERR_SELFCHECK : ORC_OK;
}

/* Entropy of one index set (LU determinant), exposed for the pins. */
int orc_entropy(const double* Sigma, int N, const int32_t* idx, int n, int64_t T_bias,
                double* H) {
  int c[ORC_MAXN];
  for (int a = 0; a < n; a++) c[a] = idx[a];
  return entropy_of(Sigma, N, c, n, T_bias, H) ? ORC_OK : ORC_ERR_SELFCHECK;
}
