"""FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg
may import this package.  The CUDA library and its Python binding never import
it; the two share no code.  The arithmetic lives in ``oracle.c`` (plain C,
FP64, OpenMP); this module compiles it, loads it with ctypes and adds the
per-order reductions, written with numpy sorts.

Paper passages followed (arXiv 2501.03381):
  * copula covariance     -- Supp. eq. gaussian_copula_covariance_estimator
  * Gaussian entropy      -- Supp. eq. gaussian_differential_entropy
  * TC, DTC, O, S         -- Methods, eqs. TC, DTC, O-info, S-info
  * enumeration / count   -- Supp. eq. comb
  * bias corrector        -- Supp. eq. bias_corrector (1/2 on the psi sum)
  * batch-level reduction -- Fig. 1A caption (per-batch custom function,
                             e.g. the minimum O), read as the fixed set
                             min/max/mean/count/count(O<0)/top-M per order.
  * greedy search         -- Methods, "Heuristics", "Greedy Algorithm"
  * simulated annealing   -- Methods, "Heuristics", "Simulated Annealing
                             Algorithm"
  * group objectives      -- Results, "Leveraging Gaussian entropy
                             estimators with batch processing" (average O
                             across datasets); Methods, "Heuristics" (the
                             searches take several datasets) and "fMRI
                             analysis" (paired Cohen's d between conditions)
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

MEASURES = ("H", "TC", "DTC", "O", "S")


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u64, i64, i32, dbl = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        vp = ctypes.c_void_p
        lib.orc_binom.restype = u64
        lib.orc_binom.argtypes = [ctypes.c_int, ctypes.c_int]
        lib.orc_count.restype = u64
        lib.orc_count.argtypes = [ctypes.c_int, vp, ctypes.c_int]
        lib.orc_rank.argtypes = [vp, i64, i64, i64, vp]
        lib.orc_ndtri.restype = dbl
        lib.orc_ndtri.argtypes = [dbl]
        lib.orc_ndtri_ratio.restype = dbl
        lib.orc_ndtri_ratio.argtypes = [dbl, dbl]
        lib.orc_copula_cov.argtypes = [vp, i64, i64, i64, vp, vp]
        lib.orc_enumerate.argtypes = [ctypes.c_int, vp, ctypes.c_int, u64, u64, ctypes.c_int, vp]
        lib.orc_unrank_ids.argtypes = [ctypes.c_int, vp, ctypes.c_int, vp, i64, ctypes.c_int, vp]
        lib.orc_measures.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, u64, u64, i64, vp, vp,
                                     ctypes.c_int]
        lib.orc_measures_ids.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, vp, i64, i64, vp, vp,
                                         ctypes.c_int]
        lib.orc_grad.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int]
        lib.orc_objective_containing.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_int, vp, ctypes.c_int]
        lib.orc_digamma.restype = dbl
        lib.orc_digamma.argtypes = [dbl]
        lib.orc_bias_eta.restype = dbl
        lib.orc_bias_eta.argtypes = [ctypes.c_int, i64]
        lib.orc_entropy.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, i64, vp]
        for f in ("orc_rank", "orc_copula_cov", "orc_enumerate", "orc_unrank_ids", "orc_measures",
                  "orc_measures_ids", "orc_grad", "orc_objective_containing", "orc_entropy"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _orders(orders) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(list(orders), dtype=np.int32))


def _check(st: int, what: str):
    if st != 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")


def binom(n: int, k: int) -> int:
    return int(_load().orc_binom(n, k))


def count(N: int, orders) -> int:
    o = _orders(orders)
    return int(_load().orc_count(N, _p(o), len(o)))


def rank(X: np.ndarray) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float64)
    T, N = X.shape
    R = np.empty((T, N), dtype=np.int32)
    _check(_load().orc_rank(_p(X), T, N, N, _p(R)), "rank")
    return R


def ndtri(u: float) -> float:
    return float(_load().orc_ndtri(float(u)))


def ndtri_ratio(num: float, den: float) -> float:
    return float(_load().orc_ndtri_ratio(float(num), float(den)))


def copula_cov(X: np.ndarray, return_z: bool = False):
    """Gaussian-copula covariance (FP64) of a T x N sample matrix."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    T, N = X.shape
    S = np.empty((N, N))
    Z = np.empty((T, N)) if return_z else None
    _check(_load().orc_copula_cov(_p(X), T, N, N, _p(Z) if Z is not None else None, _p(S)),
           "copula_cov")
    return (S, Z) if return_z else S


def enumerate_subsets(N: int, orders, id_begin: int = 0, id_end: int | None = None) -> np.ndarray:
    """Subsets by lexicographic successor, one row per id, padded with -1."""
    o = _orders(orders)
    if id_end is None:
        id_end = count(N, o)
    kmax = int(max(o))
    out = np.empty((id_end - id_begin, kmax), dtype=np.int8)
    _check(_load().orc_enumerate(N, _p(o), len(o), id_begin, id_end, kmax, _p(out)), "enumerate")
    return out


def unrank_ids(N: int, orders, ids) -> np.ndarray:
    """Subsets of the listed ids by the counting unrank, padded with -1."""
    o = _orders(orders)
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.uint64))
    kmax = int(max(o))
    out = np.empty((len(ids), kmax), dtype=np.int8)
    _check(_load().orc_unrank_ids(N, _p(o), len(o), _p(ids), len(ids), kmax, _p(out)), "unrank")
    return out


def measures(Sigma: np.ndarray, orders, id_begin: int = 0, id_end: int | None = None,
             T_bias: int = 0, nthreads: int = 0):
    """Per-nplet (H, TC, DTC, O, S) as a 5 x n FP64 array, and not-PD flags."""
    S = np.ascontiguousarray(Sigma, dtype=np.float64)
    N = S.shape[0]
    o = _orders(orders)
    if id_end is None:
        id_end = count(N, o)
    n = id_end - id_begin
    out = np.empty((5, n))
    flags = np.empty(n, dtype=np.uint8)
    _check(_load().orc_measures(_p(S), N, _p(o), len(o), id_begin, id_end, T_bias, _p(out),
                                _p(flags), nthreads), "measures")
    return out, flags


def measures_ids(Sigma: np.ndarray, orders, ids, T_bias: int = 0, nthreads: int = 0):
    """Per-nplet measures of the listed global ids (5 x len(ids))."""
    S = np.ascontiguousarray(Sigma, dtype=np.float64)
    N = S.shape[0]
    o = _orders(orders)
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.uint64))
    out = np.empty((5, len(ids)))
    flags = np.empty(len(ids), dtype=np.uint8)
    _check(_load().orc_measures_ids(_p(S), N, _p(o), len(o), _p(ids), len(ids), T_bias, _p(out),
                                    _p(flags), nthreads), "measures_ids")
    return out, flags


def grad(Sigma: np.ndarray, orders, measure: str = "O", nthreads: int = 0) -> np.ndarray:
    """Analytic dL/dSigma of L = sum over nplets of one measure (N x N)."""
    S = np.ascontiguousarray(Sigma, dtype=np.float64)
    N = S.shape[0]
    o = _orders(orders)
    G = np.empty((N, N))
    _check(_load().orc_grad(_p(S), N, _p(o), len(o), MEASURES.index(measure), _p(G), nthreads),
           "grad")
    return G


def objective_containing(Sigma: np.ndarray, orders, measure: str, i: int, j: int,
                         nthreads: int = 0) -> float:
    S = np.ascontiguousarray(Sigma, dtype=np.float64)
    N = S.shape[0]
    o = _orders(orders)
    out = np.empty(1)
    _check(_load().orc_objective_containing(_p(S), N, _p(o), len(o), MEASURES.index(measure),
                                            i, j, _p(out), nthreads), "objective_containing")
    return float(out[0])


def fd_grad_entry(Sigma: np.ndarray, orders, measure: str, i: int, j: int,
                  h: float = 1e-6) -> float:
    """Central finite difference of L in the symmetric direction E_ij + E_ji
    (E_ii on the diagonal).  Equals 2 G_ij off the diagonal and G_ii on it."""
    S = np.array(Sigma, dtype=np.float64)
    Sp, Sm = S.copy(), S.copy()
    Sp[i, j] += h
    Sm[i, j] -= h
    if i != j:
        Sp[j, i] += h
        Sm[j, i] -= h
    fp = objective_containing(Sp, orders, measure, i, j)
    fm = objective_containing(Sm, orders, measure, i, j)
    return (fp - fm) / (2.0 * h)


def digamma(x: float) -> float:
    return float(_load().orc_digamma(float(x)))


def bias_eta(m: int, T: int) -> float:
    return float(_load().orc_bias_eta(int(m), int(T)))


def entropy(Sigma: np.ndarray, idx, T_bias: int = 0) -> float:
    S = np.ascontiguousarray(Sigma, dtype=np.float64)
    i = np.ascontiguousarray(np.asarray(idx, dtype=np.int32))
    out = np.empty(1)
    _check(_load().orc_entropy(_p(S), S.shape[0], _p(i), len(i), T_bias, _p(out)), "entropy")
    return float(out[0])


def order_of_ids(N: int, orders, ids) -> np.ndarray:
    """Order k of each global id (ids enumerate the orders in list order)."""
    o = list(orders)
    offs = np.cumsum([0] + [binom(N, k) for k in o])
    ids = np.asarray(ids, dtype=np.uint64)
    slot = np.searchsorted(offs[1:], ids, side="right")
    return np.asarray(o)[slot], slot


def reduce_per_order(N: int, orders, vals: np.ndarray, ids: np.ndarray, notpd: np.ndarray,
                     top_m: int = 256):
    """Per-order reduction records from per-nplet values (Fig. 1A caption:
    a function applied per batch, e.g. the minimum O).  For each order and
    measure: min / max with the smallest id on ties, mean as a long-double sum
    over the count, the count of O < 0, and the top-M largest and smallest O
    ordered by (value, id).  Nplets marked not-PD are excluded."""
    ids = np.asarray(ids, dtype=np.uint64)
    ks, slots = order_of_ids(N, orders, ids)
    recs = []
    for s, k in enumerate(orders):
        sel = (slots == s) & (notpd == 0)
        v = vals[:, sel]
        i = ids[sel]
        rec = {"k": int(k), "count": int(sel.sum()),
               "n_not_pd": int(((slots == s) & (notpd != 0)).sum())}
        if rec["count"] == 0:
            recs.append(rec)
            continue
        rec["min"], rec["argmin"], rec["max"], rec["argmax"], rec["mean"] = [], [], [], [], []
        for m in range(5):
            x = v[m]
            order_min = np.lexsort((i, x))
            order_max = np.lexsort((i, -x))
            rec["min"].append(float(x[order_min[0]]))
            rec["argmin"].append(int(i[order_min[0]]))
            rec["max"].append(float(x[order_max[0]]))
            rec["argmax"].append(int(i[order_max[0]]))
            rec["mean"].append(float(np.sum(x.astype(np.longdouble)) / len(x)))
        o = v[3]
        rec["neg_O"] = int((o < 0).sum())
        hi = np.lexsort((i, -o))[:top_m]
        lo = np.lexsort((i, o))[:top_m]
        rec["top_hi_val"], rec["top_hi_id"] = o[hi].copy(), i[hi].copy()
        rec["top_lo_val"], rec["top_lo_id"] = o[lo].copy(), i[lo].copy()
        recs.append(rec)
    return recs


def subset_rank(N: int, members) -> int:
    """Lexicographic rank of a sorted k-subset among all k-subsets of N
    (Supp. eq. comb; rank = C(N,k) - 1 - sum_i C(N-1-c_i, k-i))."""
    k = len(members)
    return math.comb(N, k) - 1 - sum(math.comb(N - 1 - c, k - i) for i, c in enumerate(members))


def greedy(Sigma, k0: int, k1: int, kappa: int, measure: str = "O",
           maximize: bool = True, objective: str | None = None):
    """Greedy search (Methods, "Heuristics", "Greedy Algorithm"), literally:
    the kappa best nplets of order k0 from an exhaustive evaluation, then for
    each next order every selected set grows by each variable it lacks, the
    distinct candidates are evaluated, and the kappa best are kept.  Best =
    largest (or smallest) value of the measure; ties by smaller lexicographic
    rank; nplets that are not positive definite are left out.  With a list of
    covariances and a group objective ("mean" or "cohen_d"), the value is that
    objective over the datasets (Methods, "Heuristics": the searches accept
    several datasets).  Returns one (members list, values array) pair per
    order k0..k1."""
    by_range, by_ids, N = _evaluator(Sigma, measure, objective)

    def pick(ids, vals, notpd, k):
        keep = notpd == 0
        ids, vals = ids[keep], vals[keep]
        key = -vals if maximize else vals
        order = np.lexsort((ids, key))[:kappa]
        sets = [tuple(int(x) for x in row) for row in unrank_ids(N, [k], ids[order])]
        return sets, vals[order]

    out = []
    vals, notpd = by_range(k0)
    sets, best = pick(np.arange(len(vals), dtype=np.uint64), vals, notpd, k0)
    out.append((sets, best))
    for k in range(k0 + 1, k1 + 1):
        cand = sorted({tuple(sorted(s + (v,))) for s in sets for v in range(N) if v not in s})
        if not cand:
            break
        ids = np.array([subset_rank(N, c) for c in cand], dtype=np.uint64)
        vals, notpd = by_ids(k, ids)
        sets, best = pick(ids, vals, notpd, k)
        out.append((sets, best))
    return out


# ------------------------------------------------------------------ simulated annealing
M64 = (1 << 64) - 1


def splitmix64(seed: int, c: int) -> int:
    """Output c (0-based) of the SplitMix64 generator seeded with `seed`:
    the finaliser of seed + (c + 1) * 0x9E3779B97F4A7C15 (mod 2^64)."""
    z = (seed + (c + 1) * 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def anneal(Sigma, k_lo: int, k_hi: int, n_chains: int, iters: int, T0: float,
           alpha: float, measure: str = "O", maximize: bool = True, seed: int = 0,
           objective: str | None = None, patience: int = 0):
    """Simulated annealing (Methods, "Heuristics", "Simulated Annealing
    Algorithm"), chain by chain, with the moves, draws and acceptance rule
    stated for thoi_anneal: draw (chain, step, slot) is SplitMix64 output
    ((chain * (iters+1) + step) * 64 + slot); integers (z * n) >> 64; uniforms
    (z >> 11) * 2^-53; accept when the energy rises, else with probability
    exp(dE / Temp); Temp = T0 at step 1 and is multiplied by alpha after
    every step.  Termination ("Termination Criteria"): after `iters` steps,
    or, when patience > 0, after the first step t with t - t_best >= patience,
    t_best being the last step that raised the best energy (0 at the start).
    With a list of covariances and a group objective the energy is that
    objective over the datasets.  Returns (final sets, final values, best
    sets, best values) with sets as sorted tuples."""
    _, by_ids, N = _evaluator(Sigma, measure, objective)
    sgn = 1.0 if maximize else -1.0

    def value(members):
        k = len(members)
        vals, notpd = by_ids(k, np.array([subset_rank(N, members)], dtype=np.uint64))
        return float("nan") if notpd[0] else float(vals[0])

    out = ([], [], [], [])
    for ch in range(n_chains):
        base = ch * (iters + 1)

        def draw(step, slot):
            return splitmix64(seed, (base + step) * 64 + slot)

        size = k_lo + ((draw(0, 0) * (k_hi - k_lo + 1)) >> 64)
        perm = list(range(N))
        for j in range(size):
            r = j + ((draw(0, 1 + j) * (N - j)) >> 64)
            perm[j], perm[r] = perm[r], perm[j]
        cur = tuple(sorted(perm[:size]))
        E = sgn * value(cur)
        best, bestE = cur, E
        T = T0
        t_best = 0
        for it in range(1, iters + 1):
            members = list(cur)
            size = len(members)
            prop = cur
            swap = k_lo == k_hi
            if not swap:
                v = (draw(it, 0) * N) >> 64
                if v not in cur and size < k_hi:
                    prop = tuple(sorted(members + [v]))
                elif v in cur and size > k_lo:
                    prop = tuple(x for x in members if x != v)
                else:
                    swap = True
            if swap and size < N:
                v = members[(draw(it, 1) * size) >> 64]
                outside = [x for x in range(N) if x not in cur]
                w = outside[(draw(it, 2) * (N - size)) >> 64]
                prop = tuple(sorted([x for x in members if x != v] + [w]))
            En = sgn * value(prop)
            if En == En:
                dE = En - E
                ok = dE > 0.0
                if not ok:
                    p = 1.0 if dE == 0.0 else math.exp(dE / T)
                    ok = (draw(it, 3) >> 11) * 2.0 ** -53 < p
                if ok:
                    cur, E = prop, En
                    if E > bestE:
                        best, bestE = cur, E
                        t_best = it
            T *= alpha
            if patience > 0 and it - t_best >= patience:
                break
        out[0].append(cur)
        out[1].append(sgn * E)
        out[2].append(best)
        out[3].append(sgn * bestE)
    return out


# ------------------------------------------------------------------ group objectives
GROUP_OBJECTIVES = ("mean", "cohen_d")


def group_objective(V: np.ndarray, notpd: np.ndarray, objective: str):
    """Group objective of one measure over D datasets, per nplet.  V and notpd
    are D x n (values and not-PD flags of each dataset).  Results,
    "Leveraging Gaussian entropy estimators with batch processing": the nplet
    with the smallest average O across datasets; Methods, "fMRI analysis":
    nplets that maximise or minimise the paired Cohen's d between two
    conditions.
      mean    : (1/D) sum_d V[d]
      cohen_d : D = 2P (P >= 2); dataset i (condition A) is paired with dataset
                P + i (condition B); delta_i = V[i] - V[P + i];
                g = mean(delta) / sd(delta), sd with the P - 1 denominator
                (Cohen's d of paired samples)
    Returns (g, bad): an nplet is excluded (bad = 1, g = NaN) when it is not
    positive definite in some dataset, or, for cohen_d, when sd(delta) = 0."""
    V = np.asarray(V, dtype=np.float64)
    bad = np.asarray(notpd).astype(bool).any(axis=0)
    if objective == "mean":
        g = V.mean(axis=0)
    elif objective == "cohen_d":
        D = V.shape[0]
        if D % 2 or D < 4:
            raise ValueError("cohen_d needs D = 2P datasets with P >= 2")
        P = D // 2
        delta = V[:P] - V[P:]
        sd = delta.std(axis=0, ddof=1)
        bad = bad | ~(sd > 0)
        with np.errstate(divide="ignore", invalid="ignore"):
            g = delta.mean(axis=0) / sd
    else:
        raise ValueError(f"unknown group objective {objective!r}")
    return np.where(bad, np.nan, g), bad.astype(np.uint8)


def _t_biases(T_bias, D: int):
    return list(T_bias) if isinstance(T_bias, (list, tuple)) else [T_bias] * D


def group_measures(Sigmas, orders, measure: str, objective: str, id_begin: int = 0,
                   id_end: int | None = None, T_bias=0, nthreads: int = 0):
    """Per-nplet group objective over the datasets' covariances (all N x N)."""
    m = MEASURES.index(measure)
    tb = _t_biases(T_bias, len(Sigmas))
    res = [measures(S, orders, id_begin, id_end, tb[d], nthreads) for d, S in enumerate(Sigmas)]
    return group_objective(np.stack([r[0][m] for r in res]), np.stack([r[1] for r in res]),
                           objective)


def group_measures_ids(Sigmas, orders, measure: str, objective: str, ids, T_bias=0,
                       nthreads: int = 0):
    """Group objective of the listed global ids."""
    m = MEASURES.index(measure)
    tb = _t_biases(T_bias, len(Sigmas))
    res = [measures_ids(S, orders, ids, tb[d], nthreads) for d, S in enumerate(Sigmas)]
    return group_objective(np.stack([r[0][m] for r in res]), np.stack([r[1] for r in res]),
                           objective)


def _evaluator(Sigma, measure: str, objective: str | None):
    """(values of every nplet of order k, values of listed ids of order k, N)
    for one covariance and a measure, or a list of covariances and a group
    objective."""
    if objective is None:
        S = np.ascontiguousarray(Sigma, dtype=np.float64)
        m = MEASURES.index(measure)

        def by_range(k):
            v, f = measures(S, [k])
            return v[m], f

        def by_ids(k, ids):
            v, f = measures_ids(S, [k], ids)
            return v[m], f

        return by_range, by_ids, S.shape[0]
    Ss = [np.ascontiguousarray(S, dtype=np.float64) for S in Sigma]
    return (lambda k: group_measures(Ss, [k], measure, objective),
            lambda k, ids: group_measures_ids(Ss, [k], measure, objective, ids), Ss[0].shape[0])
