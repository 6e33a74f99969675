"""FP64 re-factor of the nplets the FP32 path flags (a small pivot or a large
inverse trace), against the FP64 oracle at 1e-10 nats: the sum-constrained
block of the planted workload, every nplet flagged on a 64-bit-mask dataset
over a ragged range, and per-order records built from re-factored values
only (reduced by radix select and by the streaming reduction)."""
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


def _lex_rank(c, N):
    # rank of the sorted tuple c among the len(c)-subsets of range(N) in
    # lexicographic order (checked against the oracle's unranking below)
    k, r, prev = len(c), 0, -1
    for i, ci in enumerate(c):
        for v in range(prev + 1, ci):
            r += math.comb(N - 1 - v, k - 1 - i)
        prev = ci
    return r


def test_synergy_block_order20_refactored_to_fp64():
    # order 20 of the planted N = 30 workload: every nplet holding the whole
    # sum-constrained block (variables 10..19) has a pivot near 1e-2 and is
    # re-factored; a sample of them must match the oracle at FP64 tolerance
    X, _ = workloads.planted30()
    S = oracle.copula_cov(X)
    rng = np.random.default_rng(8)
    syn = list(range(10, 20))
    rest = [v for v in range(30) if v not in syn]
    picks = {tuple(sorted(syn + [int(v) for v in rng.choice(rest, 10, replace=False)]))
             for _ in range(400)}
    picks = sorted(picks)
    ids = np.array([_lex_rank(p, 30) for p in picks], dtype=np.uint64)
    np.testing.assert_array_equal(oracle.unrank_ids(30, [20], ids)[:, :20], np.array(picks))
    free = np.sort(rng.choice(math.comb(30, 20), 400, replace=False)).astype(np.uint64)
    with P.Context(torch.as_tensor(X, device="cuda"), out_f64=True) as c:
        out, st = c.measures([20])
        got = out[:, torch.as_tensor(ids.astype(np.int64), device="cuda")].cpu().numpy()
        got_free = out[:, torch.as_tensor(free.astype(np.int64), device="cuda")].cpu().numpy()
    assert st.n_refactored >= math.comb(20, 10)
    ref, _ = oracle.measures_ids(S, [20], ids)
    np.testing.assert_allclose(got, ref, rtol=0, atol=TOL64)
    ref_free, _ = oracle.measures_ids(S, [20], free)
    np.testing.assert_allclose(got_free, ref_free, rtol=0, atol=TOL32)


def test_all_flagged_wide_masks_ragged_range():
    # N = 36 (64-bit masks), every nplet flagged (trace bound below 1), a
    # range that starts and ends inside two orders
    rng = np.random.default_rng(12)
    S = workloads.random_corr(rng, 36)
    orders = [5, 6]
    n5 = math.comb(36, 5)
    a, b = n5 - 2500, n5 + 3500
    ref, _ = oracle.measures(S, orders, a, b)
    with P.Context(Sigma=S, out_f64=True, trace_tau=0.5) as c:
        out, st = c.measures(orders, a, b)
    assert st.n_refactored == b - a
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=TOL64)


@pytest.mark.parametrize("mode", ["auto", "stored"])
def test_all_flagged_records_match_oracle(mode):
    # per-order records of orders whose whole FP32 pass is flagged: every
    # value comes from the FP64 re-factor, reduced by the radix select (auto)
    # or the streaming reduction (stored)
    X, _ = workloads.fmri_like()
    orders = [2, 9, 10, 19, 20]
    S = oracle.copula_cov(X)
    vals, fl = oracle.measures(S, orders)
    ids = np.arange(vals.shape[1], dtype=np.uint64)
    ref = oracle.reduce_per_order(20, orders, vals, ids, fl, top_m=64)
    with P.Context(torch.as_tensor(X, device="cuda"), trace_tau=0.5, top_m=64,
                   records_mode=mode) as c:
        (recs, hi, lo), st = c.measures(orders, reduction="per_order")
    assert st.n_refactored == vals.shape[1]
    for q, e in enumerate(ref):
        r = recs[q]
        assert int(r["count"]) == e["count"] + e["n_not_pd"]
        assert int(r["n_refactored"]) == math.comb(20, orders[q])
        np.testing.assert_allclose(r["min"], e["min"], rtol=0, atol=TOL64)
        np.testing.assert_allclose(r["max"], e["max"], rtol=0, atol=TOL64)
        np.testing.assert_allclose(r["mean"], e["mean"], rtol=0, atol=TOL64)
        n = int(r["top_count"])
        assert n == min(64, e["count"])
        np.testing.assert_allclose(hi[q]["value"][:n], e["top_hi_val"][:n], rtol=0, atol=TOL64)
        np.testing.assert_allclose(lo[q]["value"][:n], e["top_lo_val"][:n], rtol=0, atol=TOL64)
