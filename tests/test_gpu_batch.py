"""Multi-dataset batching (many datasets of uneven N and T through one graph
of batched launches) against the oracle and against one context at a time."""
import math

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
import paper_2501_03381_gb300 as P  # noqa: E402

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-4


def _ctx(X=None, **kw):
    if X is not None:
        return P.Context(torch.as_tensor(X, device="cuda"), **kw)
    return P.Context(**kw)


def _dataset(N, T, seed):
    rng = np.random.default_rng(seed)
    S = workloads.random_corr(rng, N)
    return np.ascontiguousarray(rng.standard_normal((T, N)) @ np.linalg.cholesky(S).T)


def _oracle_records(X, kmin, kmax, top_m):
    """The oracle's per-order records over orders kmin..min(kmax, N)."""
    N = X.shape[1]
    S = oracle.copula_cov(X)
    orders = list(range(kmin, min(kmax, N) + 1))
    vals, fl = oracle.measures(S, orders)
    ids = np.arange(vals.shape[1], dtype=np.uint64)
    return S, orders, oracle.reduce_per_order(N, orders, vals, ids, fl, top_m=top_m)


def _check_against_oracle(recs, hi, lo, S, orders, ref, tol, top_m, kmin, kmax):
    for q, k in enumerate(range(kmin, kmax + 1)):
        r = recs[q]
        assert int(r["k"]) == k
        if k not in orders:
            assert int(r["count"]) == 0 and int(r["top_count"]) == 0
            continue
        e = ref[orders.index(k)]
        assert int(r["count"]) == e["count"] + e["n_not_pd"]
        np.testing.assert_allclose(r["min"], e["min"], atol=tol)
        np.testing.assert_allclose(r["max"], e["max"], atol=tol)
        np.testing.assert_allclose(r["mean"], e["mean"], atol=tol)
        ids = np.concatenate([r["argmin"], r["argmax"]]).astype(np.uint64)
        vals, _ = oracle.measures_ids(S, orders, ids)
        for m in range(5):
            assert abs(vals[m, m] - e["min"][m]) <= tol
            assert abs(vals[m, 5 + m] - e["max"][m]) <= tol
        n = int(r["top_count"])
        assert n == min(top_m, e["count"])
        h, l_ = hi[q][:n], lo[q][:n]
        np.testing.assert_allclose(h["value"], e["top_hi_val"][:n], atol=tol)
        np.testing.assert_allclose(l_["value"], e["top_lo_val"][:n], atol=tol)
        tv, _ = oracle.measures_ids(S, orders, np.concatenate([h["id"], l_["id"]]))
        np.testing.assert_allclose(tv[3], np.concatenate([h["value"], l_["value"]]), atol=tol)


# uneven (N, T): narrow and wide masks, orders above some datasets' N
SMALL_SET = [(10, 300, 11), (13, 1700, 12), (17, 450, 13), (6, 900, 14), (21, 1200, 15)]


def test_batch_records_match_oracle():
    Xs = [_dataset(N, T, s) for N, T, s in SMALL_SET]
    kmin, kmax, top_m = 3, 7, 24
    ctxs = [_ctx(X, top_m=top_m) for X in Xs]
    try:
        res, st = P.thoi_batch_measures([c.h for c in ctxs], kmin, kmax, top_m=top_m)
        assert st.launches > 0
        for X, (recs, hi, lo) in zip(Xs, res):
            S, orders, ref = _oracle_records(X, kmin, kmax, top_m)
            _check_against_oracle(recs, hi, lo, S, orders, ref, TOL32, top_m, kmin, kmax)
        assert st.nplets == sum(oracle.count(X.shape[1], range(kmin, min(kmax, X.shape[1]) + 1))
                                for X in Xs)
    finally:
        for c in ctxs:
            c.close()


def test_batch_wide_masks_match_oracle():
    # N > 32 switches every dataset of the batch to 64-bit masks
    Xs = [_dataset(34, 800, 21), _dataset(12, 400, 22)]
    kmin, kmax, top_m = 2, 4, 16
    ctxs = [_ctx(X, top_m=top_m) for X in Xs]
    try:
        res, _ = P.thoi_batch_measures([c.h for c in ctxs], kmin, kmax, top_m=top_m)
        for X, (recs, hi, lo) in zip(Xs, res):
            S, orders, ref = _oracle_records(X, kmin, kmax, top_m)
            _check_against_oracle(recs, hi, lo, S, orders, ref, TOL32, top_m, kmin, kmax)
    finally:
        for c in ctxs:
            c.close()


def test_batch_forced_refactor_reaches_fp64_tolerance():
    # trace_tau below 1 flags every nplet: all values come from the batched
    # FP64 re-factor and its list reduction
    Xs = [_dataset(N, T, s) for N, T, s in SMALL_SET[:4]]
    kmin, kmax, top_m = 3, 6, 8
    ctxs = [_ctx(X, top_m=top_m, trace_tau=0.5) for X in Xs]
    try:
        res, st = P.thoi_batch_measures([c.h for c in ctxs], kmin, kmax, top_m=top_m)
        assert st.n_refactored == st.nplets
        for X, (recs, hi, lo) in zip(Xs, res):
            S, orders, ref = _oracle_records(X, kmin, kmax, top_m)
            _check_against_oracle(recs, hi, lo, S, orders, ref, TOL64, top_m, kmin, kmax)
            for q, k in enumerate(range(kmin, kmax + 1)):
                if k <= X.shape[1]:
                    assert int(recs[q]["n_refactored"]) == math.comb(X.shape[1], k)
    finally:
        for c in ctxs:
            c.close()


def _records_equal(a, b, mean_atol=1e-7):
    (ra, ha, la), (rb, hb, lb) = a, b
    for q in range(len(ra)):
        for f in ("k", "count", "count_neg_O", "n_refactored", "n_not_pd", "top_count"):
            assert int(ra[q][f]) == int(rb[q][f]), f
        for f in ("min", "max", "argmin", "argmax"):
            np.testing.assert_array_equal(ra[q][f], rb[q][f])
        # the sums behind the means are per-block FP32 (compensated) sums
        # combined in FP64; another tiling changes them by rounding only
        np.testing.assert_allclose(ra[q]["mean"], rb[q]["mean"], rtol=0, atol=mean_atol)
        n = int(ra[q]["top_count"])
        for x, y in ((ha[q], hb[q]), (la[q], lb[q])):
            np.testing.assert_array_equal(x["id"][:n], y["id"][:n])
            np.testing.assert_array_equal(x["value"][:n], y["value"][:n])


def test_batch_matches_single_contexts():
    # uneven datasets of the 64-dataset workload's distribution: the batch
    # evaluates every nplet with the same arithmetic as one context at a time,
    # so every extreme, id and top entry is identical; means differ only by
    # the order of summation
    Xs = workloads.multi(6, 3000)
    kmin, kmax, top_m = 3, 8, 32
    ctxs = [_ctx(X, top_m=top_m) for X in Xs]
    try:
        res, st = P.thoi_batch_measures([c.h for c in ctxs], kmin, kmax, top_m=top_m)
        tot = 0
        for c, X, got in zip(ctxs, Xs, res):
            N = X.shape[1]
            orders = list(range(kmin, min(kmax, N) + 1))
            (recs, hi, lo), _ = c.measures(orders, reduction="per_order")
            nq = len(orders)
            _records_equal((got[0][:nq], got[1][:nq], got[2][:nq]), (recs, hi, lo))
            for q in range(nq, kmax - kmin + 1):
                assert int(got[0][q]["count"]) == 0
            tot += sum(math.comb(N, k) for k in orders)
        assert st.nplets == tot
    finally:
        for c in ctxs:
            c.close()


def test_batch_graph_replay_and_cache_invalidation():
    Xa, Xb, Xc = (_dataset(14, 600, 31), _dataset(15, 700, 32), _dataset(15, 900, 33))
    kmin, kmax, top_m = 3, 6, 16
    ca, cb = _ctx(Xa, top_m=top_m), _ctx(Xb, top_m=top_m)
    first, _ = P.thoi_batch_measures([ca.h, cb.h], kmin, kmax, top_m=top_m)
    again, _ = P.thoi_batch_measures([ca.h, cb.h], kmin, kmax, top_m=top_m)
    for x, y in zip(first, again):
        _records_equal(x, y, mean_atol=0)
    # a new context (possibly at the old one's address) must not reuse the
    # destroyed context's graph
    cb.close()
    cc = _ctx(Xc, top_m=top_m)
    try:
        res, _ = P.thoi_batch_measures([ca.h, cc.h], kmin, kmax, top_m=top_m)
        S, orders, ref = _oracle_records(Xc, kmin, kmax, top_m)
        _check_against_oracle(*res[1], S, orders, ref, TOL32, top_m, kmin, kmax)
        _records_equal(res[0], first[0], mean_atol=0)
    finally:
        ca.close()
        cc.close()


def test_batch_device_output_buffer():
    Xs = [_dataset(N, T, s) for N, T, s in SMALL_SET[:3]]
    kmin, kmax, top_m = 3, 5, 4
    ctxs = [_ctx(X, top_m=top_m) for X in Xs]
    try:
        host, _ = P.thoi_batch_measures([c.h for c in ctxs], kmin, kmax, top_m=top_m)
        per = P.thoi_records_bytes(kmax - kmin + 1, top_m)
        buf = torch.zeros(per * len(Xs), dtype=torch.uint8, device="cuda")
        dev, _ = P.thoi_batch_measures([c.h for c in ctxs], kmin, kmax, top_m=top_m, out=buf)
        for x, y in zip(host, dev):
            _records_equal(x, y, mean_atol=0)
    finally:
        for c in ctxs:
            c.close()


def test_batch_flag_overflow_reports_workspace():
    # every nplet flagged, room for 4 per slot: the status word reports the
    # overflow (no device fault, no partial result claimed)
    Xs = [_dataset(12, 500, 41), _dataset(11, 500, 42)]
    ctxs = [_ctx(X, top_m=4, trace_tau=0.5, flag_capacity=4) for X in Xs]
    try:
        with pytest.raises(P.ThoiError) as ei:
            P.thoi_batch_measures([c.h for c in ctxs], 3, 5, top_m=4)
        assert ei.value.name == "THOI_ERR_WORKSPACE"
    finally:
        for c in ctxs:
            c.close()


@pytest.mark.parametrize("case", ["orders_above_20", "fp64"])
def test_batch_sequential_paths_match_single(case):
    # orders above the register kernels and the FP64 path go through one
    # context at a time; the output layout is the same
    if case == "orders_above_20":
        Xs = [_dataset(22, 800, 51), _dataset(12, 400, 52)]
        kmin, kmax, kw = 19, 22, {}
    else:
        Xs = [_dataset(12, 800, 53), _dataset(9, 400, 54)]
        kmin, kmax, kw = 3, 10, {"precision": "f64"}
    top_m = 8
    ctxs = [_ctx(X, top_m=top_m, **kw) for X in Xs]
    try:
        res, _ = P.thoi_batch_measures([c.h for c in ctxs], kmin, kmax, top_m=top_m)
        for c, X, got in zip(ctxs, Xs, res):
            orders = list(range(kmin, min(kmax, X.shape[1]) + 1))
            if not orders:
                assert all(int(r["count"]) == 0 for r in got[0])
                continue
            (recs, hi, lo), _ = c.measures(orders, reduction="per_order")
            nq = len(orders)
            _records_equal((got[0][:nq], got[1][:nq], got[2][:nq]), (recs, hi, lo), mean_atol=0)
    finally:
        for c in ctxs:
            c.close()


# ------------------------------------------------------------------ the 64-dataset workload at full size
def _records_by_ids(S, N, orders, recs, hi, lo, tol):
    """Every reported extreme and top-list id of every order re-evaluated by
    the oracle at its id: the value stored beside it must match within tol."""
    ids, want = [], []
    for q, k in enumerate(orders):
        r = recs[q]
        for m in range(5):
            ids += [int(r["argmin"][m]), int(r["argmax"][m])]
            want += [(m, float(r["min"][m])), (m, float(r["max"][m]))]
        n = int(r["top_count"])
        for lst in (hi[q][:n], lo[q][:n]):
            ids += [int(x) for x in lst["id"]]
            want += [(3, float(v)) for v in lst["value"]]
    vals, fl = oracle.measures_ids(S, orders, np.array(ids, dtype=np.uint64))
    assert not fl.any()
    got = np.array([v for _, v in want])
    ref = np.array([vals[m, j] for j, (m, _) in enumerate(want)])
    err = np.abs(got - ref).max()
    assert err <= tol, err


def test_multi64_full_size_matches_single_contexts_and_oracle():
    # the 64-dataset workload exactly as the bench runs it (N ~ U{10..40},
    # T ~ U{200..2000}, orders 3..min(N, 8), top-256 lists, one replayed
    # graph): records identical to one context at a time with the built-in
    # (dense) kernels, which share the batch kernel's arithmetic, and every
    # reported id's value confirmed by the oracle
    Xs, ords = workloads.multi64()
    kmin, kmax, top_m = 3, 8, 256
    ctxs = [_ctx(X, top_m=top_m, autotune=False) for X in Xs]
    try:
        res, st = P.thoi_batch_measures([c.h for c in ctxs], kmin, kmax, top_m=top_m)
        assert st.nplets == sum(oracle.count(X.shape[1], o) for X, o in zip(Xs, ords))
        for X, o, c, got in zip(Xs, ords, ctxs, res):
            (recs, hi, lo), _ = c.measures(o, reduction="per_order")
            nq = len(o)
            _records_equal((got[0][:nq], got[1][:nq], got[2][:nq]), (recs, hi, lo))
            for q in range(nq, kmax - kmin + 1):  # orders above N_d
                assert int(got[0][q]["count"]) == 0
            S = oracle.copula_cov(X)
            _records_by_ids(S, X.shape[1], o, got[0][:nq], got[1][:nq], got[2][:nq], TOL32)
    finally:
        for c in ctxs:
            c.close()


def test_multi64_full_size_forced_refactor():
    # every nplet of the 64 datasets flagged (trace_tau below 1): all values
    # from the batched FP64 re-factor, confirmed by the oracle at 1e-10
    Xs, ords = workloads.multi64()
    kmin, kmax, top_m = 3, 8, 16
    ctxs = [_ctx(X, top_m=top_m, trace_tau=0.5,
                 flag_capacity=max(math.comb(X.shape[1], k) for k in o))
            for X, o in zip(Xs, ords)]
    try:
        res, st = P.thoi_batch_measures([c.h for c in ctxs], kmin, kmax, top_m=top_m)
        assert st.n_refactored == st.nplets
        for X, o, (recs, hi, lo) in zip(Xs, ords, res):
            nq = len(o)
            for q, k in enumerate(o):
                assert int(recs[q]["n_refactored"]) == math.comb(X.shape[1], k)
            S = oracle.copula_cov(X)
            _records_by_ids(S, X.shape[1], o, recs[:nq], hi[:nq], lo[:nq], TOL64)
    finally:
        for c in ctxs:
            c.close()
