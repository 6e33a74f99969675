"""Fused per-order records (the reduction inside the FP32 nplet kernels:
sample bounds, per-thread sums, a candidate list, a certified merge) against
the records formed from stored per-nplet values and against the oracle.

Both modes evaluate every nplet with the same FP32 kernel, and the extremes
and top lists of both come from the same reduction arithmetic on the same
FP32 values, so they must agree exactly; the means differ only by the order
of summation, and the count of O < 0 only on nplets whose O rounds to zero
differently in the two reductions."""
import math
import os
import tempfile

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
import paper_2501_03381_gb300 as P  # noqa: E402

pytestmark = pytest.mark.gpu

TOL32 = 1e-4


def _records(X, orders, mode, id_begin=0, id_end=None, tune=False, **kw):
    with P.Context(torch.as_tensor(X, device="cuda"), records_mode=mode, **kw) as c:
        if tune:
            P.thoi_autotune(c.h, min(orders), max(orders),
                            os.path.join(tempfile.mkdtemp(), "tune.json"))
        res, st = c.measures(orders, id_begin, id_end, reduction="per_order")
    return res, st


def _same_records(a, b, mean_atol=1e-6, neg_slack=2):
    (ra, ha, la), (rb, hb, lb) = a, b
    for q in range(len(ra)):
        for f in ("k", "count", "n_refactored", "n_not_pd", "top_count"):
            assert int(ra[q][f]) == int(rb[q][f]), (q, f)
        for f in ("min", "max", "argmin", "argmax"):
            np.testing.assert_array_equal(ra[q][f], rb[q][f], err_msg=f"order slot {q} {f}")
        np.testing.assert_allclose(ra[q]["mean"], rb[q]["mean"], rtol=0, atol=mean_atol)
        assert abs(int(ra[q]["count_neg_O"]) - int(rb[q]["count_neg_O"])) <= neg_slack
        n = int(ra[q]["top_count"])
        for x, y in ((ha[q], hb[q]), (la[q], lb[q])):
            np.testing.assert_array_equal(x["id"][:n], y["id"][:n])
            np.testing.assert_array_equal(x["value"][:n], y["value"][:n])


@pytest.mark.parametrize("tune", [False, True])
def test_fused_matches_stored_fmri_like(tune):
    # every order of the fMRI-shaped workload, with the built-in (dense)
    # kernels and with the autotuner's (prefix-shared and lane-group) ones
    X, orders = workloads.fmri_like()
    fused, st = _records(X, orders, "fused", tune=tune)
    stored, _ = _records(X, orders, "stored", tune=tune)
    assert st.fused_retries == 0
    _same_records(fused, stored)


def test_fused_matches_oracle_fmri_like():
    X, orders = workloads.fmri_like()
    S = oracle.copula_cov(X)
    vals, fl = oracle.measures(S, orders)
    ids = np.arange(vals.shape[1], dtype=np.uint64)
    ref = oracle.reduce_per_order(20, orders, vals, ids, fl, top_m=256)
    (recs, hi, lo), st = _records(X, orders, "fused")
    assert st.fused_retries == 0
    for q, (r, e) in enumerate(zip(recs, ref)):
        assert int(r["count"]) == e["count"] + e["n_not_pd"]
        np.testing.assert_allclose(r["min"], e["min"], atol=TOL32)
        np.testing.assert_allclose(r["max"], e["max"], atol=TOL32)
        np.testing.assert_allclose(r["mean"], e["mean"], atol=TOL32)
        n = int(r["top_count"])
        assert n == min(256, e["count"])
        np.testing.assert_allclose(hi[q]["value"][:n], e["top_hi_val"][:n], atol=TOL32)
        np.testing.assert_allclose(lo[q]["value"][:n], e["top_lo_val"][:n], atol=TOL32)
        got = np.concatenate([r["argmin"], r["argmax"], hi[q]["id"][:n], lo[q]["id"][:n]])
        tv, _ = oracle.measures_ids(S, orders, got.astype(np.uint64))
        np.testing.assert_allclose(tv[np.arange(5), np.arange(5)], r["min"], atol=TOL32)
        np.testing.assert_allclose(tv[np.arange(5), 5 + np.arange(5)], r["max"], atol=TOL32)
        np.testing.assert_allclose(tv[3, 10:], np.concatenate([hi[q]["value"][:n],
                                                               lo[q]["value"][:n]]), atol=TOL32)


def _force_shape(h, k, prefix, chunk, path):
    import json
    props = torch.cuda.get_device_properties(0)
    ent = {"gpu": props.name, "sms": props.multi_processor_count, "k": k, "wide": 0,
           "lanes": 1, "chunk": chunk, "blocks_per_sm": 0, "prefix": prefix}
    with open(path, "w") as fh:
        fh.write("[\n" + json.dumps(ent) + "\n]\n")
    P.thoi_autotune(h, k, k, path)


@pytest.mark.parametrize("prefix,chunk", [(0, 8), (1, 1), (3, 1), (5, 2)])
def test_fused_single_orders_need_no_retry(prefix, chunk, tmp_path):
    # one small order per request (its candidate list is then sized to the
    # order itself), with the dense kernel and with prefix kernels, which
    # take their work dynamically and may leave most candidates to a few
    # blocks: entries go on to other segments of the list instead of
    # forcing the stored-value retry
    X, _ = workloads.fmri_like()
    S = oracle.copula_cov(X)
    ks = (3, 4, 5, 6, 7, 8)
    with P.Context(torch.as_tensor(X, device="cuda"), records_mode="fused") as c:
        try:
            for k in ks:
                _force_shape(c.h, k, prefix, chunk, str(tmp_path / f"s{k}.json"))
                vals, fl = oracle.measures(S, [k])
                ids = np.arange(vals.shape[1], dtype=np.uint64)
                e = oracle.reduce_per_order(20, [k], vals, ids, fl, top_m=256)[0]
                (recs, hi, lo), st = c.measures([k], reduction="per_order")
                assert st.fused_retries == 0, k
                r = recs[0]
                assert int(r["count"]) == e["count"] + e["n_not_pd"]
                np.testing.assert_allclose(r["min"], e["min"], atol=TOL32)
                np.testing.assert_allclose(r["max"], e["max"], atol=TOL32)
                n = int(r["top_count"])
                assert n == min(256, e["count"])
                np.testing.assert_allclose(hi[0]["value"][:n], e["top_hi_val"][:n], atol=TOL32)
                np.testing.assert_allclose(lo[0]["value"][:n], e["top_lo_val"][:n], atol=TOL32)
        finally:
            # the shape cache is process-wide: leave the dense default behind
            for k in ks:
                _force_shape(c.h, k, 0, 8, str(tmp_path / f"d{k}.json"))


@pytest.mark.parametrize("top_m", [0, 1, 7, 1024])
def test_fused_top_m_edges_and_subranges(top_m):
    X, orders = workloads.fmri_like()
    # a ragged sub-range across three orders, and the whole request
    a = math.comb(20, 3) + math.comb(20, 4) + 12345
    b = a + math.comb(20, 5) + math.comb(20, 6) // 3
    for lo_, hi_ in ((a, b), (0, None)):
        fused, st = _records(X, orders, "fused", lo_, hi_, top_m=top_m)
        stored, _ = _records(X, orders, "stored", lo_, hi_, top_m=top_m)
        _same_records(fused, stored)


def test_fused_falls_back_when_bounds_admit_everything():
    # Sigma = I: every nplet has O = TC = DTC = 0 exactly, so every nplet lies
    # at the sample's bounds, the candidate list overflows, and the request is
    # repeated with stored values; the records are the closed forms
    orders = [9, 10, 11]
    with P.Context(Sigma=np.eye(20), records_mode="fused") as c:
        (recs, hi, lo), st = c.measures(orders, reduction="per_order")
    assert st.fused_retries == 1
    for q, k in enumerate(orders):
        assert int(recs[q]["count"]) == math.comb(20, k)
        np.testing.assert_allclose(recs[q]["min"][1:], 0.0, atol=1e-6)
        np.testing.assert_allclose(recs[q]["max"][1:], 0.0, atol=1e-6)
        # ties go to the smallest id: the first nplets of the order
        assert int(recs[q]["argmin"][3]) == sum(math.comb(20, kk) for kk in orders[:q])
        np.testing.assert_allclose(recs[q]["mean"][0], k * 1.4189385332046727, atol=1e-5)


def test_fused_refactored_nplets_and_wide_masks():
    # N = 34 (64-bit masks), an ill-conditioned pair of columns so that some
    # nplets go to the FP64 re-factor list, fused against stored
    rng = np.random.default_rng(91)
    S = workloads.random_corr(rng, 34)
    X = rng.standard_normal((900, 34)) @ np.linalg.cholesky(S).T
    X[:, 7] = X[:, 3] + 1e-3 * rng.standard_normal(900)
    orders = [3, 4, 5]
    fused, st = _records(X, orders, "fused")
    stored, st2 = _records(X, orders, "stored")
    assert st.n_refactored == st2.n_refactored > 0
    _same_records(fused, stored)


@pytest.mark.parametrize("top_m", [0, 1, 256])
def test_select_reductions_match_streaming(top_m):
    # automatic mode on orders below the fused threshold: the stored FP32
    # values and the FP64 re-factor lists reduced by radix select, against the
    # streaming reductions of the stored mode (identical extremes and lists)
    rng = np.random.default_rng(5)
    S = workloads.random_corr(rng, 20)
    X = rng.standard_normal((700, 20)) @ np.linalg.cholesky(S).T
    X[:, 11] = X[:, 2] - X[:, 5] + 2e-3 * rng.standard_normal(700)
    orders = [3, 4, 7, 10, 13, 19, 20]
    auto, st = _records(X, orders, "auto", top_m=top_m)
    stored, st2 = _records(X, orders, "stored", top_m=top_m)
    assert st.fused_retries == 0
    assert st.n_refactored == st2.n_refactored > 0
    _same_records(auto, stored, mean_atol=1e-6, neg_slack=0)


def test_select_falls_back_on_ties_in_auto_mode():
    # Sigma = I: every O is exactly 0, so more than the select's survivors tie
    # at the M-th value; the request is repeated with the streaming reductions
    orders = [9, 10, 11]
    with P.Context(Sigma=np.eye(20)) as c:
        (recs, hi, lo), st = c.measures(orders, reduction="per_order")
    assert st.fused_retries == 1
    for q, k in enumerate(orders):
        base = sum(math.comb(20, kk) for kk in orders[:q])
        assert int(recs[q]["count"]) == math.comb(20, k)
        np.testing.assert_array_equal(hi[q]["id"][:256], base + np.arange(256))
        np.testing.assert_array_equal(lo[q]["id"][:256], base + np.arange(256))
