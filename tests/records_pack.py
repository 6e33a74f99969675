"""Packs the oracle's per-order reductions into the byte layout of the
library's record output (thoi_order_record x n, then the top lists), so that
host-side record logic can be checked on the CPU against the oracle."""
import numpy as np

import paper_2501_03381_gb300 as P


def pack(recs, top_m: int) -> np.ndarray:
    n = len(recs)
    R = np.zeros(n, dtype=P.RECORD_DTYPE)
    T = np.zeros((n, 2, top_m), dtype=P.TOP_DTYPE)
    T["id"] = np.uint64(~np.uint64(0))
    for q, e in enumerate(recs):
        R[q]["k"] = e["k"]
        R[q]["count"] = e["count"] + e["n_not_pd"]
        R[q]["n_not_pd"] = e["n_not_pd"]
        if e["count"] == 0:
            R[q]["argmin"] = R[q]["argmax"] = np.uint64(~np.uint64(0))
            continue
        R[q]["min"], R[q]["max"], R[q]["mean"] = e["min"], e["max"], e["mean"]
        R[q]["argmin"], R[q]["argmax"] = e["argmin"], e["argmax"]
        R[q]["count_neg_O"] = e["neg_O"]
        c = min(top_m, e["count"])
        R[q]["top_count"] = c
        T[q, 0, :c]["value"], T[q, 0, :c]["id"] = e["top_hi_val"][:c], e["top_hi_id"][:c]
        T[q, 1, :c]["value"], T[q, 1, :c]["id"] = e["top_lo_val"][:c], e["top_lo_id"][:c]
    return np.concatenate([R.view(np.uint8), T.reshape(-1).view(np.uint8)])


def assert_same(a, b, n_orders: int, top_m: int, mean_atol: float = 1e-12):
    ra, ha, la = P.parse_records(a, n_orders, top_m)
    rb, hb, lb = P.parse_records(b, n_orders, top_m)
    for q in range(n_orders):
        for f in ("k", "count", "count_neg_O", "n_refactored", "n_not_pd", "top_count"):
            assert int(ra[q][f]) == int(rb[q][f]), (q, f)
        for f in ("min", "max", "argmin", "argmax"):
            np.testing.assert_array_equal(ra[q][f], rb[q][f])
        np.testing.assert_allclose(ra[q]["mean"], rb[q]["mean"], rtol=0, atol=mean_atol)
        n = int(ra[q]["top_count"])
        for x, y in ((ha[q], hb[q]), (la[q], lb[q])):
            np.testing.assert_array_equal(x["id"][:n], y["id"][:n])
            np.testing.assert_array_equal(x["value"][:n], y["value"][:n])
