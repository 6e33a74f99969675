"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

None of these checks re-types the oracle's own formula: each compares the
oracle with a closed form, a brute-force computation written differently, a
library routine for a special case, or an invariant.  A dropped term, a wrong
sign or a transposed index in the oracle fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.special

import oracle
import workloads

LOG2PIE_HALF = 1.4189385332046727  # entropy of N(0,1), the 1.4189 of the padding section


# ---------------------------------------------------------------- helpers
def cofactor_det(A):
    """Determinant by Laplace expansion along the first row (tiny n only)."""
    n = len(A)
    if n == 0:
        return 1.0
    if n == 1:
        return A[0][0]
    s = 0.0
    for j in range(n):
        minor = [row[:j] + row[j + 1:] for row in A[1:]]
        s += (-1) ** j * A[0][j] * cofactor_det(minor)
    return s


def entropy_bf(S, idx):
    if len(idx) == 0:
        return 0.0
    sub = [[S[a][b] for b in idx] for a in idx]
    return 0.5 * (len(idx) * math.log(2 * math.pi * math.e) + math.log(cofactor_det(sub)))


def measures_bf(S, idx):
    """TC/DTC/O/S from eqs. TC, DTC, O-info, S-info with cofactor determinants."""
    k = len(idx)
    HS = entropy_bf(S, idx)
    singles = [entropy_bf(S, [i]) for i in idx]
    loo = [entropy_bf(S, [i for i in idx if i != j]) for j in idx]
    tc = sum(singles) - HS
    dtc = HS - sum(HS - h for h in loo)
    return np.array([HS, tc, dtc, tc - dtc, tc + dtc])


def rand_spd(rng, n, ridge=0.3):
    W = rng.standard_normal((n, n))
    A = W @ W.T + ridge * np.eye(n)
    return A


# ---------------------------------------------------------------- counts
@pytest.mark.parametrize("N", [3, 5, 10, 20, 30, 40, 60])
def test_count_formula(N):
    # Supp. eq. comb: sum_{k=3}^{N} C(N,k) = 2^N - 1 - N - N(N-1)/2
    assert oracle.count(N, range(3, N + 1)) == 2 ** N - 1 - N - N * (N - 1) // 2


def test_count_c4():
    assert oracle.count(60, [3, 4, 5]) == 34220 + 487635 + 5461512 == 5983367


# ---------------------------------------------------------------- enumeration
@pytest.mark.parametrize("N", [1, 2, 4, 6])
def test_enumeration_bruteforce(N):
    orders = list(range(1, N + 1))
    got = oracle.enumerate_subsets(N, orders)
    exp = []
    for k in orders:
        subs = [tuple(i for i in range(N) if (m >> i) & 1) for m in range(1 << N)
                if bin(m).count("1") == k]
        exp += sorted(subs)  # lexicographic order of the sorted tuple
    assert len(got) == len(exp)
    for row, e in zip(got, exp):
        assert tuple(int(x) for x in row if x >= 0) == e


def test_enumeration_itertools_n12():
    N, orders = 12, [5, 3, 7]  # caller's order list is honoured
    got = oracle.enumerate_subsets(N, orders)
    exp = [c for k in orders for c in itertools.combinations(range(N), k)]
    assert len(got) == len(exp)
    for row, e in zip(got, exp):
        assert tuple(int(x) for x in row if x >= 0) == e


def test_unrank_counting_matches_successor():
    N, orders = 14, list(range(1, 15))
    walk = oracle.enumerate_subsets(N, orders)
    ids = np.arange(len(walk), dtype=np.uint64)
    un = oracle.unrank_ids(N, orders, ids)
    assert np.array_equal(walk, un)


def test_unrank_n30_spot():
    N, orders = 30, list(range(3, 31))
    rng = np.random.default_rng(5)
    total = oracle.count(N, orders)
    ids = np.unique(np.concatenate([rng.integers(0, total, 2000, dtype=np.uint64),
                                    np.array([0, total - 1], dtype=np.uint64)]))
    sub = oracle.unrank_ids(N, orders, ids)
    offs = np.cumsum([0] + [math.comb(N, k) for k in orders])
    for gid, row in zip(ids, sub):
        s = int(np.searchsorted(offs[1:], gid, side="right"))
        k = orders[s]
        r = int(gid) - int(offs[s])
        c = tuple(int(x) for x in row if x >= 0)
        assert len(c) == k and list(c) == sorted(set(c))
        # lexicographic rank of c by counting the subsets that precede it
        rk, prev = 0, -1
        for i, ci in enumerate(c):
            for x in range(prev + 1, ci):
                rk += math.comb(N - 1 - x, k - 1 - i)
            prev = ci
        assert rk == r


# ---------------------------------------------------------------- measures
def test_identity_all_zero():
    # Sigma = I: H = k * 1/2 log(2 pi e); all dependence measures vanish
    for k in range(1, 7):
        out, fl = oracle.measures(np.eye(6), [k])
        assert not fl.any()
        np.testing.assert_allclose(out[0], k * LOG2PIE_HALF, rtol=0, atol=1e-13)
        np.testing.assert_allclose(out[1:], 0.0, rtol=0, atol=1e-13)


def _equicorr_logdet(k, rho):
    return (k - 1) * math.log(1 - rho) + math.log(1 + (k - 1) * rho)


@pytest.mark.parametrize("rho", [-0.08, 0.1, 0.5, 0.9])
def test_equicorrelated_closed_form(rho):
    N = 9
    S = np.full((N, N), rho) + (1 - rho) * np.eye(N)
    for k in range(2, N + 1):
        out, _ = oracle.measures(S, [k], 0, 1)
        ld = _equicorr_logdet(k, rho)
        tc = -0.5 * ld
        dtc = 0.5 * (k * _equicorr_logdet(k - 1, rho) - (k - 1) * ld)
        np.testing.assert_allclose(out[:, 0], [0.5 * (k * math.log(2 * math.pi * math.e) + ld),
                                               tc, dtc, tc - dtc, tc + dtc], rtol=0, atol=1e-12)


def test_pair_mi_equivalence():
    # eqs. MI-tc and MI-dtc coincide for two variables: O = 0, TC = DTC = MI
    rng = np.random.default_rng(1)
    for _ in range(20):
        a, b = rng.uniform(0.2, 3.0, 2)
        rho = rng.uniform(-0.99, 0.99)
        S = np.array([[a, rho * math.sqrt(a * b)], [rho * math.sqrt(a * b), b]])
        out, _ = oracle.measures(S, [2])
        mi = -0.5 * math.log(1 - rho * rho)
        np.testing.assert_allclose(out[1:4, 0], [mi, mi, 0.0], rtol=0, atol=1e-12)


def test_tc_dtc_nonnegative():
    rng = np.random.default_rng(2)
    for _ in range(5):
        S = rand_spd(rng, 8)
        out, _ = oracle.measures(S, range(2, 9))
        assert (out[1] > -1e-12).all() and (out[2] > -1e-12).all()


def _rsys(n, c):
    S = np.full((n + 1, n + 1), c * c)
    S[np.arange(n), np.arange(n)] = c * c + 1
    S[:n, n] = S[n, :n] = c
    S[n, n] = 1.0
    return S


def _ssys(n, c):
    S = np.eye(n + 1)
    S[:n, n] = S[n, :n] = c
    S[n, n] = n * c * c + 1
    return S


def _closed_measures(logdet, var, idx):
    """TC/DTC/O from a closed-form logdet(idx) (entropy definitions)."""
    k = len(idx)
    L = logdet(idx)
    tc = 0.5 * (sum(math.log(var(i)) for i in idx) - L)
    dtc = 0.5 * L - sum(0.5 * L - 0.5 * logdet([i for i in idx if i != j]) for j in idx)
    return tc, dtc, tc - dtc


@pytest.mark.parametrize("c", [0.5, 1.0])
def test_r_and_s_systems(c):
    n = 6
    # R-system (tail-to-tail, PGM section): det of m X's = 1 + m c^2, with Y: 1
    R = _rsys(n, c)
    r_ld = lambda idx: 0.0 if n in idx else math.log(1 + len(idx) * c * c)
    r_var = lambda i: 1.0 if i == n else c * c + 1
    # S-system (head-to-head): det of m X's = 1, with Y: 1 + (n - m) c^2
    S = _ssys(n, c)
    s_ld = lambda idx: math.log(1 + (n - (len(idx) - 1)) * c * c) if n in idx else 0.0
    s_var = lambda i: n * c * c + 1 if i == n else 1.0
    orders = list(range(3, n + 2))
    outR, _ = oracle.measures(R, orders)
    outS, _ = oracle.measures(S, orders)
    subs = oracle.enumerate_subsets(n + 1, orders)
    for q, row in enumerate(subs):
        idx = [int(x) for x in row if x >= 0]
        np.testing.assert_allclose(outR[1:4, q], _closed_measures(r_ld, r_var, idx), atol=1e-12)
        np.testing.assert_allclose(outS[1:4, q], _closed_measures(s_ld, s_var, idx), atol=1e-12)
        # sign convention of eq. O-info: redundancy > 0, synergy < 0
        assert outR[3, q] > 1e-9
        if n in idx:
            assert outS[3, q] < -1e-9
        else:
            assert abs(outS[3, q]) < 1e-12


def test_additivity_independent_blocks():
    # independent blocks: every measure of A u B is the sum over the blocks
    rng = np.random.default_rng(3)
    A, B = rand_spd(rng, 3), rand_spd(rng, 4)
    S = np.zeros((7, 7))
    S[:3, :3], S[3:, 3:] = A, B
    full, _ = oracle.measures(S, [7])
    a, _ = oracle.measures(A, [3])
    b, _ = oracle.measures(B, [4])
    np.testing.assert_allclose(full[:, 0], a[:, 0] + b[:, 0], atol=1e-12)


@pytest.mark.parametrize("N", [3, 4, 5, 6])
def test_bruteforce_cofactor(N):
    rng = np.random.default_rng(10 + N)
    S = rand_spd(rng, N)
    orders = list(range(1, N + 1))
    out, fl = oracle.measures(S, orders)
    subs = oracle.enumerate_subsets(N, orders)
    Sl = S.tolist()
    for q, row in enumerate(subs):
        idx = [int(x) for x in row if x >= 0]
        np.testing.assert_allclose(out[:, q], measures_bf(Sl, idx), rtol=1e-11, atol=1e-11)


def test_padding_identity():
    # padding Sigma_S with an independent identity block adds (n-k) * 1.4189
    rng = np.random.default_rng(4)
    A = rand_spd(rng, 4)
    P = np.eye(7)
    P[:4, :4] = A
    h_pad = oracle.entropy(P, range(7))
    h = oracle.entropy(A, range(4))
    assert abs(h_pad - (h + 3 * LOG2PIE_HALF)) < 1e-12


def _golden(name):
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    vals = {}
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                key, val = line.split()
                vals[key] = float(val)
    return vals


def test_padding_constant_as_printed():
    # the printed 1.4189 (four decimals) against the oracle's entropy of one
    # unit-variance normal, and the padding identity with the printed value
    # within its rounding
    h1 = _golden("padding_entropy.txt")["h_unit_normal"]
    assert round(oracle.entropy(np.eye(1), [0]), 4) == h1
    rng = np.random.default_rng(8)
    A = rand_spd(rng, 3)
    for n_pad in (1, 4, 9):
        P = np.eye(3 + n_pad)
        P[:3, :3] = A
        err = oracle.entropy(P, range(3 + n_pad)) - (oracle.entropy(A, range(3)) + n_pad * h1)
        assert abs(err) <= n_pad * 5e-5


def test_not_pd_marked():
    S = np.eye(5)
    S[0, 1] = S[1, 0] = 1.0  # duplicated variable: singular
    out, fl = oracle.measures(S, [2, 3])
    subs = oracle.enumerate_subsets(5, [2, 3])
    for q, row in enumerate(subs):
        bad = 0 in row and 1 in row
        assert bool(fl[q]) == bad
        assert np.isnan(out[:, q]).all() == bad


def test_measures_ids_match_range():
    rng = np.random.default_rng(6)
    S = rand_spd(rng, 12)
    orders = list(range(3, 13))
    full, _ = oracle.measures(S, orders)
    ids = rng.choice(full.shape[1], 300, replace=False).astype(np.uint64)
    part, _ = oracle.measures_ids(S, orders, ids)
    np.testing.assert_array_equal(part, full[:, ids.astype(np.int64)])


# ---------------------------------------------------------------- copula front end
def test_ndtri_library_and_roundtrip():
    us = np.concatenate([np.linspace(1e-4, 1 - 1e-4, 997), [0.5, 1 / 2001, 2000 / 2001]])
    for u in us:
        z = oracle.ndtri(u)
        assert abs(z - scipy.special.ndtri(u)) < 2e-14 * max(1.0, abs(z))
        if u <= 0.5:
            # the best double z misses u by at most phi(z) * ulp(z) / 2, plus
            # the rounding of erfc itself (relative, a few ulp)
            phi = math.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)
            tol = phi * math.ulp(z) + 6e-16 * u
            assert abs(0.5 * math.erfc(-z / math.sqrt(2)) - u) <= tol
    assert oracle.ndtri(0.5) == 0.0
    T = 999
    for r in range(T):
        assert oracle.ndtri_ratio(r + 1, T + 1) == -oracle.ndtri_ratio(T - r, T + 1)


def test_rank_bruteforce_with_ties():
    rng = np.random.default_rng(7)
    T, N = 40, 5
    X = rng.integers(-3, 4, size=(T, N)).astype(np.float64)  # many ties
    X[3, 0], X[9, 0] = -0.0, 0.0
    R = oracle.rank(X)
    for j in range(N):
        for t in range(T):
            exp = sum(1 for s in range(T) if X[s, j] < X[t, j]) + \
                  sum(1 for s in range(t) if X[s, j] == X[t, j])
            assert R[t, j] == exp
        assert sorted(R[:, j]) == list(range(T))


def test_rank_rejects_nan():
    X = np.ones((5, 2))
    X[2, 1] = np.nan
    with pytest.raises(RuntimeError):
        oracle.rank(X)


def test_copula_invariance_under_monotone_maps():
    rng = np.random.default_rng(8)
    X = rng.standard_normal((300, 6))
    S = oracle.copula_cov(X)
    for f in (np.exp, lambda x: x ** 3, lambda x: 2.5 * x - 7.0):
        assert np.array_equal(oracle.copula_cov(f(X)), S)


def test_copula_cov_vs_numpy():
    rng = np.random.default_rng(9)
    X = rng.standard_normal((500, 7))
    S, Z = oracle.copula_cov(X, return_z=True)
    R = oracle.rank(X)
    Zs = scipy.special.ndtri((R + 1) / (X.shape[0] + 1))
    np.testing.assert_allclose(Z, Zs, rtol=0, atol=1e-13)
    np.testing.assert_allclose(S, np.cov(Z, rowvar=False), rtol=0, atol=1e-14)
    # every column is a permutation of the same table: equal diagonals, zero mean
    assert np.ptp(np.diag(S)) < 1e-14
    assert abs(Z.mean()) < 1e-15


def test_column_permutation_permutes_results():
    rng = np.random.default_rng(11)
    X = rng.standard_normal((200, 6))
    perm = np.array([3, 0, 5, 1, 4, 2])
    S = oracle.copula_cov(X)
    Sp = oracle.copula_cov(X[:, perm])
    np.testing.assert_array_equal(Sp, S[np.ix_(perm, perm)])
    out, _ = oracle.measures(S, [6])
    outp, _ = oracle.measures(Sp, [6])
    np.testing.assert_allclose(out, outp, atol=1e-13)


# ---------------------------------------------------------------- bias corrector
def test_digamma_library():
    for x in [0.3, 1.0, 2.5, 7.0, 24.5, 999.5]:
        assert abs(oracle.digamma(x) - scipy.special.digamma(x)) < 1e-13 * max(1, abs(x))


def test_bias_eta_monte_carlo():
    # E[1/2 logdet(sample cov)] - 1/2 logdet(Sigma) = eta_m (Wishart moment);
    # the reading with 1/2 on the digamma sum, not the printed one
    rng = np.random.default_rng(12)
    m, T, reps = 3, 50, 6000
    A = rand_spd(rng, m)
    L = np.linalg.cholesky(A)
    vals = np.empty(reps)
    for r in range(reps):
        Xs = rng.standard_normal((T, m)) @ L.T
        vals[r] = 0.5 * np.linalg.slogdet(np.cov(Xs, rowvar=False))[1]
    mc = vals.mean() - 0.5 * np.linalg.slogdet(A)[1]
    se = vals.std() / math.sqrt(reps)
    eta = oracle.bias_eta(m, T)
    assert abs(mc - eta) < 5 * se
    printed = 0.5 * m * math.log(2 / (T - 1)) + sum(scipy.special.digamma((T - j) / 2)
                                                     for j in range(1, m + 1))
    assert abs(mc - printed) > 50 * se


def test_bias_applied_per_entropy():
    rng = np.random.default_rng(13)
    S = rand_spd(rng, 5)
    T = 300
    raw, _ = oracle.measures(S, [4])
    cor, _ = oracle.measures(S, [4], T_bias=T)
    e = [oracle.bias_eta(m, T) for m in range(6)]
    k = 4
    np.testing.assert_allclose(cor[0], raw[0] - e[k], atol=1e-12)
    np.testing.assert_allclose(cor[1], raw[1] - k * e[1] + e[k], atol=1e-12)
    np.testing.assert_allclose(cor[2], raw[2] + (k - 1) * e[k] - k * e[k - 1], atol=1e-12)


# ---------------------------------------------------------------- gradient
@pytest.mark.parametrize("measure", ["H", "TC", "DTC", "O", "S"])
def test_grad_fd(measure):
    rng = np.random.default_rng(14)
    N = 7
    A = rand_spd(rng, N, ridge=1.0)
    d = np.sqrt(np.diag(A))
    S = A / np.outer(d, d)
    orders = [3, 4, 5]
    G = oracle.grad(S, orders, measure)
    assert np.allclose(G, G.T, atol=1e-10)
    for i in range(N):
        for j in range(i, N):
            fd = oracle.fd_grad_entry(S, orders, measure, i, j, h=1e-6)
            an = G[i, j] if i == j else 2 * G[i, j]
            assert abs(fd - an) < 2e-6 * max(1.0, abs(an)), (i, j, fd, an)


# ---------------------------------------------------------------- reductions
def test_reduce_per_order_bruteforce():
    rng = np.random.default_rng(15)
    N, orders = 9, [3, 4, 5]
    S = rand_spd(rng, N)
    vals, flags = oracle.measures(S, orders)
    # plant exact ties to exercise the smallest-id rule
    vals[3, 10] = vals[3, 20] = vals[3, 5]
    ids = np.arange(vals.shape[1], dtype=np.uint64)
    recs = oracle.reduce_per_order(N, orders, vals, ids, flags, top_m=7)
    off = 0
    for s, k in enumerate(orders):
        n = math.comb(N, k)
        rec = recs[s]
        assert rec["count"] == n
        for m in range(5):
            best_min = best_max = None
            for q in range(off, off + n):  # pure-python scan, first occurrence wins
                v = vals[m, q]
                if best_min is None or v < vals[m, best_min]:
                    best_min = q
                if best_max is None or v > vals[m, best_max]:
                    best_max = q
            assert rec["argmin"][m] == best_min and rec["argmax"][m] == best_max
            assert abs(rec["mean"][m] - sum(vals[m, off:off + n]) / n) < 1e-12
        pairs = sorted(((vals[3, q], q) for q in range(off, off + n)), key=lambda p: (-p[0], p[1]))
        assert [int(q) for _, q in pairs[:7]] == [int(x) for x in rec["top_hi_id"]]
        pairs = sorted(((vals[3, q], q) for q in range(off, off + n)), key=lambda p: (p[0], p[1]))
        assert [int(q) for _, q in pairs[:7]] == [int(x) for x in rec["top_lo_id"]]
        assert rec["neg_O"] == int((vals[3, off:off + n] < 0).sum())
        off += n


# ---------------------------------------------------------------- planted structure
def test_planted_signs():
    import workloads
    X, _ = workloads.planted30()
    S = oracle.copula_cov(X)
    red = np.array([[0, 1, 2, 3, 4]])
    syn = np.array([[10, 11, 12, 13, 19]])
    for c, sign in ((red, 1), (syn, -1)):
        k = c.shape[1]
        # global id of a subset of one order: its lexicographic rank
        rk, prev = 0, -1
        for i, ci in enumerate(c[0]):
            for x in range(prev + 1, ci):
                rk += math.comb(30 - 1 - x, k - 1 - i)
            prev = ci
        out, _ = oracle.measures_ids(S, [k], [rk])
        assert np.sign(out[3, 0]) == sign


# ------------------------------------------------------------------ greedy search (Methods, "Greedy Algorithm")
def test_subset_rank_inverts_enumeration():
    for N in (1, 5, 9):
        for k in range(1, N + 1):
            subs = oracle.enumerate_subsets(N, [k])
            got = [oracle.subset_rank(N, [int(x) for x in row]) for row in subs]
            assert got == list(range(len(subs)))


@pytest.mark.parametrize("measure,maximize", [("O", True), ("O", False), ("S", True), ("TC", False)])
def test_greedy_covering_kappa_equals_exhaustive(measure, maximize):
    # with kappa at least the number of subsets of every order, the selection
    # holds every set, so each order's result is the exhaustive top list
    rng = np.random.default_rng(31)
    S = workloads.random_corr(rng, 8)
    m = oracle.MEASURES.index(measure)
    res = oracle.greedy(S, 2, 7, 70, measure, maximize)
    for (sets, vals), k in zip(res, range(2, 8)):
        v, _ = oracle.measures(S, [k])
        ids = np.arange(v.shape[1], dtype=np.uint64)
        key = -v[m] if maximize else v[m]
        order = np.lexsort((ids, key))
        ref = [tuple(int(x) for x in r) for r in oracle.unrank_ids(8, [k], ids[order])]
        assert sets == ref
        np.testing.assert_array_equal(vals, v[m][order])


def test_greedy_selection_properties():
    rng = np.random.default_rng(32)
    S = workloads.random_corr(rng, 12)
    res = oracle.greedy(S, 3, 8, 10, "O", False)
    prev = None
    for (sets, vals), k in zip(res, range(3, 9)):
        assert all(len(s) == k for s in sets)
        assert len(set(sets)) == len(sets) == 10
        assert np.all(np.diff(vals) >= 0)  # best (smallest) first
        if prev is not None:
            # every selected set grew from a set selected one order below
            assert all(any(set(p) < set(s) for p in prev) for s in sets)
        prev = sets


# ------------------------------------------------------------------ simulated annealing (Methods, "Simulated Annealing Algorithm")
def test_splitmix64_published_outputs():
    # the first outputs of SplitMix64 seeded with 0, as published with the generator
    assert [oracle.splitmix64(0, i) for i in range(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_anneal_zero_temperature_only_climbs():
    # with a vanishing temperature a worse move is never taken, so the final
    # set of every chain is its best one
    S = workloads.random_corr(np.random.default_rng(51), 12)
    fin, fval, best, bval = oracle.anneal(S, 3, 8, 6, 40, 1e-300, 0.9, "O", True, seed=3)
    assert fin == best
    np.testing.assert_array_equal(fval, bval)


def test_anneal_start_and_ranges():
    S = workloads.random_corr(np.random.default_rng(52), 10)
    fin, fval, best, bval = oracle.anneal(S, 4, 7, 20, 0, 1.0, 0.9, "S", False, seed=9)
    assert fin == best
    for s in fin:
        assert 4 <= len(s) <= 7 and len(set(s)) == len(s) and all(0 <= x < 10 for x in s)
    fin, _, best, bval = oracle.anneal(S, 5, 5, 10, 50, 0.3, 0.95, "O", False, seed=1)
    assert all(len(s) == 5 for s in fin + best)
    # minimising: the best value is no worse than the final one
    assert all(b <= f + 1e-15 for b, f in zip(bval, oracle.anneal(S, 5, 5, 10, 50, 0.3, 0.95, "O",
                                                                   False, seed=1)[1]))


# Three-state system for the acceptance and cooling pins: N = 3 variables and
# sets of exactly two (k_lo = k_hi = 2), so the states are the three pairs.
# The energy is TC, which for a pair is the mutual information
# -1/2 log(1 - rho^2).  A swap replaces one of the two members (probability
# 1/2 each) by the one variable left out, so the proposal is symmetric, and
# the law of a chain after n steps follows from the 3 x 3 Metropolis
# transition matrices alone: a move is taken when the energy does not fall,
# else with probability exp(dE / Temp), Temp = T0 alpha^(t-1) at step t.
RHO3 = {(0, 1): 0.8, (0, 2): 0.5, (1, 2): 0.3}
STATES3 = [(0, 1), (0, 2), (1, 2)]


def _sigma3():
    S = np.eye(3)
    for (a, b), r in RHO3.items():
        S[a, b] = S[b, a] = r
    return S


def _energies3():
    return np.array([-0.5 * math.log(1.0 - RHO3[s] ** 2) for s in STATES3])


def _law3(temps, accept=lambda dE, T: 1.0 if dE >= 0 else math.exp(dE / T)):
    E = _energies3()
    p = np.full(3, 1.0 / 3.0)  # the start: a uniformly drawn pair
    for T in temps:
        M = np.zeros((3, 3))
        for a in range(3):
            for b in range(3):
                if a != b:
                    M[a, b] = 0.5 * accept(E[b] - E[a], T)
            M[a, a] = 1.0 - M[a].sum()
        p = p @ M
    return p


def _final_freq3(chains, iters, T0, alpha, seed):
    fin, _, _, _ = oracle.anneal(_sigma3(), 2, 2, chains, iters, T0, alpha, "TC", True, seed=seed)
    return np.array([sum(1 for s in fin if s == st) for st in STATES3]) / chains


def _band_dev(freq, p, n):
    # largest deviation in standard errors of a multinomial proportion
    return float(np.max(np.abs(freq - p) / np.sqrt(p * (1.0 - p) / n)))


def test_anneal_constant_temperature_reaches_boltzmann_law():
    # alpha = 1: the chain's law tends to exp(E / Temp) / Z (detailed balance
    # of the Metropolis rule with a symmetric proposal); after 30 steps the
    # exact law is that one to rounding, and the oracle's chains follow it
    T, iters, chains = 0.2, 30, 3000
    E = _energies3()
    boltz = np.exp(E / T) / np.exp(E / T).sum()
    law = _law3([T] * iters)
    np.testing.assert_allclose(law, boltz, rtol=0, atol=1e-9)
    freq = _final_freq3(chains, iters, T, 1.0, seed=2025)
    assert _band_dev(freq, law, chains) < 4.5
    # the acceptance as printed, exp(-dE / Temp) >= 1, takes every move: the
    # law would be uniform, far outside the band
    printed = _law3([T] * iters, accept=lambda dE, T: min(1.0, math.exp(-dE / T)))
    assert _band_dev(printed, law, chains) > 9.0


def test_anneal_cooling_schedule():
    # alpha < 1: step t runs at T0 alpha^(t-1).  Cooling before the first
    # step, or not cooling, gives laws many standard errors away.
    T0, alpha, iters, chains = 0.5, 0.4, 3, 4000
    law = _law3([T0 * alpha ** t for t in range(iters)])
    freq = _final_freq3(chains, iters, T0, alpha, seed=77)
    assert _band_dev(freq, law, chains) < 4.5
    early = _law3([T0 * alpha ** (t + 1) for t in range(iters)])
    flat = _law3([T0] * iters)
    assert _band_dev(early, law, chains) > 9.0 and _band_dev(flat, law, chains) > 9.0


def test_anneal_patience_stops_after_no_improvement():
    # Termination Criteria: with patience p the chain stops after the first
    # step t at which the best energy has not risen for p steps.  Chain 0's
    # draws do not depend on the step count, so its best value after t steps
    # comes from fixed-length runs; the stopping step follows, and the early
    # stopped run must equal the fixed run of that length.
    S = workloads.random_corr(np.random.default_rng(53), 8)
    iters, p, stopped = 40, 4, 0
    for seed in range(8):
        runs = [oracle.anneal(S, 3, 5, 1, t, 0.05, 0.97, "O", True, seed=seed)
                for t in range(iters + 1)]
        best = [r[3][0] for r in runs]
        t_best, stop = 0, iters
        for t in range(1, iters + 1):
            if best[t] > best[t - 1]:
                t_best = t
            if t - t_best >= p:
                stop = t
                break
        stopped += stop < iters
        got = oracle.anneal(S, 3, 5, 1, iters, 0.05, 0.97, "O", True, seed=seed, patience=p)
        assert got[0] == runs[stop][0] and got[2] == runs[stop][2]
        assert got[1] == runs[stop][1] and got[3] == runs[stop][3]
    assert stopped >= 4


# ------------------------------------------------------------------ group objectives (Results,
# "Leveraging Gaussian entropy estimators with batch processing"; Methods, "fMRI analysis")
def _equicorr(N, rho):
    return np.full((N, N), rho) + (1 - rho) * np.eye(N)


def test_group_mean_equicorrelated_closed_form():
    # the mean TC over datasets of equicorrelated systems, against the closed
    # form TC = -1/2 log det of each, averaged by hand
    rhos = [0.1, 0.35, -0.05, 0.6, 0.8]
    N = 7
    Ss = [_equicorr(N, r) for r in rhos]
    for k in range(2, N + 1):
        g, bad = oracle.group_measures(Ss, [k], "TC", "mean")
        assert not bad.any()
        ref = sum(-0.5 * _equicorr_logdet(k, r) for r in rhos) / len(rhos)
        np.testing.assert_allclose(g, ref, rtol=0, atol=1e-13)


def test_group_mean_of_copies_is_the_measure():
    rng = np.random.default_rng(61)
    S = workloads.random_corr(rng, 9)
    v, _ = oracle.measures(S, [3, 4, 5])
    g, bad = oracle.group_measures([S] * 5, [3, 4, 5], "O", "mean")
    assert not bad.any()
    np.testing.assert_allclose(g, v[3], rtol=1e-14, atol=1e-15)


def test_group_cohen_d_matches_paired_t_statistic():
    # the paired Cohen's d is the paired t statistic over sqrt(P); the t
    # statistic comes from scipy's paired t test
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(62)
    P, N = 6, 8
    Ss = [workloads.random_corr(rng, N) for _ in range(2 * P)]
    for meas in ("O", "S", "TC"):
        g, bad = oracle.group_measures(Ss, [3, 5], meas, "cohen_d")
        assert not bad.any()
        m = oracle.MEASURES.index(meas)
        V = np.stack([oracle.measures(S, [3, 5])[0][m] for S in Ss])
        t = stats.ttest_rel(V[:P], V[P:], axis=0).statistic
        np.testing.assert_allclose(g, t / math.sqrt(P), rtol=1e-12, atol=1e-13)


def test_group_cohen_d_equicorrelated_closed_form():
    # condition A and B are equicorrelated with subject-specific rho: each
    # difference of TC is a closed form; d from Python's statistics module
    import statistics
    ra = [0.2, 0.3, 0.25, 0.5]
    rb = [0.1, 0.22, 0.2, 0.3]
    N, k = 6, 4
    Ss = [_equicorr(N, r) for r in ra + rb]
    g, _ = oracle.group_measures(Ss, [k], "TC", "cohen_d")
    dl = [0.5 * (_equicorr_logdet(k, b) - _equicorr_logdet(k, a)) for a, b in zip(ra, rb)]
    ref = statistics.mean(dl) / statistics.stdev(dl)
    np.testing.assert_allclose(g, ref, rtol=1e-12)


def test_group_cohen_d_invariants():
    rng = np.random.default_rng(63)
    P, N = 5, 8
    A = [workloads.random_corr(rng, N) for _ in range(P)]
    B = [workloads.random_corr(rng, N) for _ in range(P)]
    g, _ = oracle.group_measures(A + B, [3, 4], "O", "cohen_d")
    # swapping the conditions flips the sign
    g2, _ = oracle.group_measures(B + A, [3, 4], "O", "cohen_d")
    np.testing.assert_allclose(g2, -g, rtol=1e-13, atol=1e-14)
    # permuting the subjects (jointly in both conditions) changes nothing
    perm = [3, 0, 4, 1, 2]
    g3, _ = oracle.group_measures([A[i] for i in perm] + [B[i] for i in perm], [3, 4], "O",
                                  "cohen_d")
    np.testing.assert_allclose(g3, g, rtol=1e-12, atol=1e-13)
    # breaking the pairing (condition B rotated) changes the value
    g4, _ = oracle.group_measures(A + B[1:] + B[:1], [3, 4], "O", "cohen_d")
    assert np.max(np.abs(g4 - g)) > 1e-3


def test_group_degenerate_and_not_pd_excluded():
    rng = np.random.default_rng(64)
    A = [workloads.random_corr(rng, 6) for _ in range(3)]
    # identical conditions: every difference is 0, sd = 0 -> excluded
    g, bad = oracle.group_measures(A + A, [3], "O", "cohen_d")
    assert bad.all() and np.isnan(g).all()
    # a rank-deficient dataset: nplets holding both copies of a variable are
    # not positive definite there, and so excluded from the group
    S = A[0].copy()
    S[5, :] = S[4, :]
    S[:, 5] = S[:, 4]
    g, bad = oracle.group_measures([A[1], S, A[2]], [3], "O", "mean")
    sets = oracle.enumerate_subsets(6, [3])
    both = np.array([4 in r and 5 in r for r in sets])
    np.testing.assert_array_equal(bad.astype(bool), both)
    assert np.isnan(g[both]).all() and np.isfinite(g[~both]).all()
    with pytest.raises(ValueError):
        oracle.group_objective(np.zeros((3, 2)), np.zeros((3, 2)), "cohen_d")


def test_group_greedy_covering_kappa_equals_exhaustive():
    rng = np.random.default_rng(65)
    Ss = [workloads.random_corr(rng, 7) for _ in range(6)]
    for obj in ("mean", "cohen_d"):
        res = oracle.greedy(Ss, 2, 6, 40, "O", False, objective=obj)
        for (sets, vals), k in zip(res, range(2, 7)):
            g, bad = oracle.group_measures(Ss, [k], "O", obj)
            ids = np.arange(len(g), dtype=np.uint64)[bad == 0]
            order = np.lexsort((ids, g[bad == 0]))
            ref = [tuple(int(x) for x in r) for r in oracle.unrank_ids(7, [k], ids[order])]
            assert sets == ref
            np.testing.assert_array_equal(vals, g[bad == 0][order])


def test_group_anneal_of_copies_matches_single():
    # the mean over copies of one dataset takes the same path, draw for draw,
    # as the single-dataset search
    S = workloads.random_corr(np.random.default_rng(66), 10)
    one = oracle.anneal(S, 3, 6, 4, 30, 0.05, 0.95, "O", True, seed=5)
    grp = oracle.anneal([S, S, S], 3, 6, 4, 30, 0.05, 0.95, "O", True, seed=5, objective="mean")
    assert one[0] == grp[0] and one[2] == grp[2]
    np.testing.assert_allclose(grp[1], one[1], rtol=1e-14)
    np.testing.assert_allclose(grp[3], one[3], rtol=1e-14)


def test_greedy_on_concatenated_r_and_s_systems():
    # the paper's redundant (R) and synergistic (S) systems side by side
    # (independent blocks): the largest O of each order lies in the R block
    # and the smallest in the S block with its common child; both values
    # have closed forms (the block measures of test_r_and_s_systems)
    import scipy.linalg
    n, c = 5, 1.0
    R, S = _rsys(n, c), _ssys(n, c)
    M = scipy.linalg.block_diag(R, S)
    r_ld = lambda idx: 0.0 if n in idx else math.log(1 + len(idx) * c * c)
    r_var = lambda i: 1.0 if i == n else c * c + 1
    s_ld = lambda idx: math.log(1 + (n - (len(idx) - 1)) * c * c) if n in idx else 0.0
    s_var = lambda i: n * c * c + 1 if i == n else 1.0
    hi = oracle.greedy(M, 3, n + 1, 4, "O", True)
    lo = oracle.greedy(M, 3, n + 1, 4, "O", False)
    for lvl, k in enumerate(range(3, n + 2)):
        blk = [list(t) for t in itertools.combinations(range(n + 1), k)]
        best_r = max(_closed_measures(r_ld, r_var, idx)[2] for idx in blk)
        best_s = min(_closed_measures(s_ld, s_var, idx)[2] for idx in blk)
        sets, vals = hi[lvl]
        assert max(sets[0]) <= n
        np.testing.assert_allclose(vals[0], best_r, rtol=0, atol=1e-12)
        sets, vals = lo[lvl]
        assert min(sets[0]) > n and 2 * n + 1 in sets[0]
        np.testing.assert_allclose(vals[0], best_s, rtol=0, atol=1e-12)
