"""Group objectives over datasets (mean of a measure; paired Cohen's d)
through the C ABI, against the oracle's group objectives.

Tolerance: every per-dataset value is within eps of the oracle (1e-4 for the
FP32 path with the FP64 re-factor, 1e-10 for the FP64 path).  The mean then
moves by at most eps.  For Cohen's d = m / s over P pairs, each difference
moves by at most 2 eps, so |dm| <= 2 eps and |ds| <= 2 eps sqrt(P / (P-1)),
and |d' - d| <= 2 eps (1 + |d| sqrt(P/(P-1))) / (s - 2 eps sqrt(P/(P-1))).
"""
import math

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
import paper_2501_03381_gb300 as P  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {"f32_fix64": 1e-4, "f64": 1e-10}


def _bound(objective, V, eps):
    """Per-nplet bound on |g_gpu - g_oracle| from the per-dataset bound eps
    (V: D x n oracle values of the measure)."""
    if objective == "mean":
        return np.full(V.shape[1], eps * (1 + 1e-9)) + 1e-13
    Pn = V.shape[0] // 2
    delta = V[:Pn] - V[Pn:]
    s = delta.std(axis=0, ddof=1)
    d = np.abs(delta.mean(axis=0) / s)
    r = math.sqrt(Pn / (Pn - 1))
    den = s - 2 * eps * r
    with np.errstate(divide="ignore", invalid="ignore"):
        b = np.where(den > 0, 2 * eps * (1 + d * r) / den, np.inf)
    return b * (1 + 1e-9) + 1e-13


def _datasets(D, N=10, T=500, base=100):
    return [workloads.plain(N, T, base + d) for d in range(D)]


def _oracle_V(Ss, orders, measure, ids=None):
    m = oracle.MEASURES.index(measure)
    if ids is None:
        res = [oracle.measures(S, orders) for S in Ss]
    else:
        res = [oracle.measures_ids(S, orders, ids) for S in Ss]
    return np.stack([r[0][m] for r in res]), np.stack([r[1] for r in res])


def _ctxs(Xs, **kw):
    return [P.Context(torch.as_tensor(X, device="cuda"), **kw) for X in Xs]


def _close(cs):
    for c in cs:
        c.close()


@pytest.mark.parametrize("precision", ["f32_fix64", "f64"])
@pytest.mark.parametrize("objective,measure", [("mean", "O"), ("mean", "S"), ("mean", "H"),
                                               ("cohen_d", "O"), ("cohen_d", "TC")])
def test_group_values_match_oracle(precision, objective, measure):
    Xs = _datasets(6)
    orders = list(range(3, 11))
    Ss = [oracle.copula_cov(X) for X in Xs]
    V, F = _oracle_V(Ss, orders, measure)
    g_ref, bad = oracle.group_objective(V, F, objective)
    assert not bad.any()
    cs = _ctxs(Xs, precision=precision)
    try:
        g, st = P.thoi_group_measures(cs, orders, measure, objective)
    finally:
        _close(cs)
    g = g.cpu().numpy()
    assert g.shape == g_ref.shape and st.nplets == 6 * g.size
    b = _bound(objective, V, TOL[precision])
    ok = np.isfinite(b)
    assert ok.mean() > 0.99
    assert np.all(np.abs(g - g_ref)[ok] <= b[ok]), np.max(np.abs(g - g_ref)[ok] / b[ok])


@pytest.mark.parametrize("precision", ["f32_fix64", "f64"])
@pytest.mark.parametrize("objective", ["mean", "cohen_d"])
def test_group_records_match_oracle(precision, objective):
    """Records against per-nplet bounds b_i (|g'_i - g_i| <= b_i): the
    reported extremes carry their ids' values, no nplet lies beyond them by
    more than its bound, the mean is within the mean bound, and the j-th entry
    of a top list lies between the j-th order statistics of g - b and g + b."""
    # O of a pair is identically 0, so the paired differences of order 2 are
    # rounding noise: Cohen's d starts at order 3
    Xs = workloads.paired(4, 10, 400, 7000) if objective == "cohen_d" else _datasets(5)
    orders = list(range(3 if objective == "cohen_d" else 2, 11))
    Ss = [oracle.copula_cov(X) for X in Xs]
    V, F = _oracle_V(Ss, orders, "O")
    g_ref, bad = oracle.group_objective(V, F, objective)
    assert not bad.any()
    b = _bound(objective, V, TOL[precision])
    top_m = 16
    ids = np.arange(g_ref.size, dtype=np.uint64)
    cs = _ctxs(Xs, precision=precision, top_m=top_m)
    try:
        (recs, hi, lo), st = P.thoi_group_measures(cs, orders, "O", objective,
                                                   kind=P.THOI_RED_PER_ORDER, top_m=top_m)
        g_dev, _ = P.thoi_group_measures(cs, orders, "O", objective)
    finally:
        _close(cs)
    g_dev = g_dev.cpu().numpy()
    slot = np.asarray(oracle.order_of_ids(10, orders, ids)[1])
    for q, r in enumerate(recs):
        sel = slot == q
        g, bq = g_ref[sel], b[sel]
        base = int(np.flatnonzero(sel)[0])
        assert int(r["k"]) == orders[q]
        assert int(r["count"]) == int(sel.sum()) and int(r["n_not_pd"]) == 0
        assert int(r["count_neg_O"]) == int(np.sum(g_dev[sel] < 0))
        for m in range(5):  # every slot carries the objective
            lo_i, hi_i = int(r["argmin"][m]) - base, int(r["argmax"][m]) - base
            assert abs(g[lo_i] - r["min"][m]) <= bq[lo_i]
            assert abs(g[hi_i] - r["max"][m]) <= bq[hi_i]
            assert np.all(r["min"][m] <= g + bq) and np.all(r["max"][m] >= g - bq)
            assert abs(r["mean"][m] - g.mean()) <= bq.mean() + 1e-12
        n = int(r["top_count"])
        assert n == min(top_m, int(sel.sum()))
        lower, upper = np.sort(g - bq)[::-1][:n], np.sort(g + bq)[::-1][:n]
        assert np.all(hi[q]["value"][:n] >= lower) and np.all(hi[q]["value"][:n] <= upper)
        lower, upper = np.sort(g - bq)[:n], np.sort(g + bq)[:n]
        assert np.all(lo[q]["value"][:n] >= lower) and np.all(lo[q]["value"][:n] <= upper)
        for lst in (hi[q], lo[q]):
            got = lst["id"][:n].astype(np.int64)
            assert len(set(got.tolist())) == n
            assert np.all(np.abs(g_ref[got] - lst["value"][:n]) <= b[got])
            # the records and the per-nplet output come from the same values
            np.testing.assert_array_equal(g_dev[got], lst["value"][:n])


def test_group_subrange_and_empty():
    # a sub-range may run other kernels than the whole orders (the prefix-
    # shared kernels need whole orders), so both are held to the oracle
    Xs = _datasets(4)
    orders = list(range(3, 11))
    Ss = [oracle.copula_cov(X) for X in Xs]
    V, F = _oracle_V(Ss, orders, "O")
    g_ref, _ = oracle.group_objective(V, F, "cohen_d")
    b = _bound("cohen_d", V, TOL["f32_fix64"])
    cs = _ctxs(Xs)
    try:
        full, _ = P.thoi_group_measures(cs, orders, "O", "cohen_d")
        part, st = P.thoi_group_measures(cs, orders, "O", "cohen_d", 100, 700)
        empty, st0 = P.thoi_group_measures(cs, orders, "O", "cohen_d", 500, 500)
    finally:
        _close(cs)
    assert part.numel() == 600 and st.nplets == 4 * 600
    assert np.all(np.abs(full.cpu().numpy() - g_ref) <= b)
    assert np.all(np.abs(part.cpu().numpy() - g_ref[100:700]) <= b[100:700])
    assert empty.numel() == 0 and st0.nplets == 0


def test_group_many_datasets_several_pieces():
    # 1024 datasets (4 distinct contexts, each used many times): the value
    # matrix holds at most 2^34 / (8 * 1024) = 2097152 nplets per piece, so
    # order 12 of N = 24 (2704156 nplets) takes two pieces or more
    Xs = _datasets(4, N=24, T=300, base=300)
    Ss = [oracle.copula_cov(X) for X in Xs]
    cs = _ctxs(Xs, top_m=32)
    Pn = 512
    A = [i % 2 for i in range(Pn)]
    B = [2 + (i % 3 == 0) for i in range(Pn)]
    try:
        for objective, sel in (("mean", [i % 4 for i in range(1024)]), ("cohen_d", A + B)):
            hs = [cs[i] for i in sel]
            g, st = P.thoi_group_measures(hs, [12], "O", objective)
            (recs, hi, lo), _ = P.thoi_group_measures(hs, [12], "O", objective,
                                                      kind=P.THOI_RED_PER_ORDER, top_m=32)
            g = g.cpu().numpy()
            n = math.comb(24, 12)
            assert g.size == n and st.nplets == 1024 * n
            rng = np.random.default_rng(5)
            ids = np.unique(np.concatenate([rng.integers(0, n, 300),
                                            [0, 2097151, 2097152, n - 1]]))
            ids = ids.astype(np.uint64)
            Vd, Fd = _oracle_V(Ss, [12], "O", ids)
            V = Vd[sel]
            g_ref, bad = oracle.group_objective(V, Fd[sel], objective)
            assert not bad.any()
            b = _bound(objective, V, 1e-4)
            np.testing.assert_array_less(np.abs(g[ids.astype(np.int64)] - g_ref), b)
            r = recs[0]
            assert int(r["count"]) == n and int(r["n_not_pd"]) == 0
            assert r["min"][3] == g.min() and r["max"][3] == g.max()
            order = np.lexsort((np.arange(n), -g))[:32]
            np.testing.assert_array_equal(hi[0]["id"][:32], order)
            np.testing.assert_array_equal(hi[0]["value"][:32], g[order])
            order = np.lexsort((np.arange(n), g))[:32]
            np.testing.assert_array_equal(lo[0]["id"][:32], order)
            assert abs(r["mean"][3] - g.mean()) <= 1e-9 * max(1.0, abs(g.mean()))
    finally:
        _close(cs)


def test_group_not_positive_definite_excluded():
    rng = np.random.default_rng(71)
    Ss = [workloads.random_corr(rng, 6) for _ in range(3)]
    S = Ss[1].copy()
    S[5, :] = S[4, :]
    S[:, 5] = S[:, 4]
    Ss[1] = S
    sets = oracle.enumerate_subsets(6, [3])
    both = np.array([4 in row and 5 in row for row in sets])
    for prec in ("f64", "f32_fix64"):
        cs = [P.Context(Sigma=x, precision=prec, top_m=4) for x in Ss]
        try:
            out = torch.full((20,), 7.0, dtype=torch.float64, device="cuda")
            with pytest.raises(P.ThoiError) as e:
                P.thoi_group_measures(cs, [3], "O", "mean", out=out)
            assert e.value.name == "THOI_ERR_NOT_PD"
            g = out.cpu().numpy()
            np.testing.assert_array_equal(np.isnan(g), both)
            buf = np.zeros(P.thoi_records_bytes(1, 4), dtype=np.uint8)
            with pytest.raises(P.ThoiError):
                P.thoi_group_measures(cs, [3], "O", "mean", kind=P.THOI_RED_PER_ORDER, out=buf,
                                      top_m=4)
            recs, _, _ = P.parse_records(buf, 1, 4)
            assert int(recs[0]["count"]) == 20 and int(recs[0]["n_not_pd"]) == int(both.sum())
        finally:
            _close(cs)


def test_group_cohen_degenerate_identical_conditions():
    Xs = _datasets(3)
    cs = _ctxs(Xs, top_m=4)
    try:
        g, _ = P.thoi_group_measures(cs + cs, [3, 4], "O", "cohen_d")
        (recs, _, _), _ = P.thoi_group_measures(cs + cs, [3, 4], "O", "cohen_d",
                                                kind=P.THOI_RED_PER_ORDER, top_m=4)
    finally:
        _close(cs)
    assert torch.isnan(g).all()
    for r in recs:
        assert int(r["n_not_pd"]) == int(r["count"]) and int(r["top_count"]) == 0


def test_group_arguments():
    Xs = _datasets(3)
    cs = _ctxs(Xs)
    other = P.Context(torch.as_tensor(workloads.plain(9, 300, 1), device="cuda"))
    try:
        for hs, obj in ((cs[:2], "cohen_d"), (cs, "cohen_d"), (cs + [other], "mean")):
            with pytest.raises(P.ThoiError) as e:
                P.thoi_group_measures(hs, [3], "O", obj)
            assert e.value.name == "THOI_ERR_INVALID_ARG"
        with pytest.raises(P.ThoiError):
            P.thoi_group_measures(cs, [3], "O", 7)
        with pytest.raises(P.ThoiError):
            P.thoi_group_greedy(cs[:2] * 1, 3, 4, 4, "O", "cohen_d")
        with pytest.raises(P.ThoiError):
            P.thoi_group_anneal(cs + [other], 3, 4, 4, 5, 1.0, 0.9, "O", "mean")
    finally:
        _close(cs)
        other.close()


def _members(mask):
    m = int(mask)
    return tuple(i for i in range(64) if m >> i & 1)


@pytest.mark.parametrize("objective,maximize", [("mean", False), ("mean", True),
                                                ("cohen_d", True), ("cohen_d", False)])
def test_group_greedy_matches_oracle(objective, maximize):
    rng = np.random.default_rng(72)
    Ss = [workloads.random_corr(rng, 12) for _ in range(6)]
    ref = oracle.greedy(Ss, 3, 7, 8, "O", maximize, objective=objective)
    cs = [P.Context(Sigma=S) for S in Ss]
    try:
        masks, values, st = P.thoi_group_greedy(cs, 3, 7, 8, "O", objective, maximize)
    finally:
        _close(cs)
    for lvl, (sets, vals) in enumerate(ref):
        n = len(sets)
        assert [_members(x) for x in masks[lvl, :n]] == sets
        np.testing.assert_allclose(values[lvl, :n], vals, rtol=0, atol=1e-9)


@pytest.mark.parametrize("objective,klo,khi", [("mean", 3, 6), ("cohen_d", 4, 4),
                                               ("cohen_d", 3, 7)])
def test_group_anneal_matches_oracle(objective, klo, khi):
    rng = np.random.default_rng(73)
    Ss = [workloads.random_corr(rng, 10) for _ in range(4)]
    ref = oracle.anneal(Ss, klo, khi, 6, 40, 0.05, 0.95, "O", True, seed=11,
                        objective=objective)
    cs = [P.Context(Sigma=S) for S in Ss]
    try:
        fm, fv, bm, bv, st = P.thoi_group_anneal(cs, klo, khi, 6, 40, 0.05, 0.95, "O",
                                                 objective, True, 11)
    finally:
        _close(cs)
    assert [_members(x) for x in fm] == ref[0]
    assert [_members(x) for x in bm] == ref[2]
    np.testing.assert_allclose(fv, ref[1], rtol=0, atol=1e-9)
    np.testing.assert_allclose(bv, ref[3], rtol=0, atol=1e-9)
    assert st.nplets == 6 * 41 * 4


def test_group_anneal_patience_matches_oracle():
    rng = np.random.default_rng(74)
    Ss = [workloads.random_corr(rng, 10) for _ in range(4)]
    ref = oracle.anneal(Ss, 3, 6, 6, 60, 0.05, 0.95, "O", True, seed=12, objective="mean",
                        patience=5)
    cs = [P.Context(Sigma=S) for S in Ss]
    try:
        fm, fv, bm, bv, _ = P.thoi_group_anneal(cs, 3, 6, 6, 60, 0.05, 0.95, "O", "mean", True,
                                                12, patience=5)
    finally:
        _close(cs)
    assert [_members(x) for x in fm] == ref[0]
    assert [_members(x) for x in bm] == ref[2]
    np.testing.assert_allclose(bv, ref[3], rtol=0, atol=1e-9)
