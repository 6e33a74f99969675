"""The entry point that allocates no device memory, checked against the
regular per-order reduction of the FP64 path.

It serves callers that cannot call cudaMalloc or cudaFree (device memory
held entirely by another allocator, or no tolerance for the synchronisation
those calls can cause).  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
import paper_2501_03381_gb300 as P  # noqa: E402

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def _regular(S, k, top_m):
    with P.Context(Sigma=S, precision="f64", top_m=top_m) as c:
        (recs, hi, lo), _ = c.measures([k], reduction="per_order")
    return recs[0], hi[0], lo[0]


@pytest.mark.parametrize("k,top_m", [(5, 16), (3, 0), (10, 7)])
def test_noalloc_matches_regular_entry_point(k, top_m):
    X, _ = workloads.small()
    S = oracle.copula_cov(X)
    ref, rhi, rlo = _regular(S, k, top_m)
    Sd = torch.as_tensor(S, device="cuda")
    for _ in range(2):  # two calls in a row share the static scratch array
        rec, hi, lo = P.thoi_order_record_noalloc(Sd, k, top_m)
        assert int(rec["k"]) == k and int(rec["count"]) == int(ref["count"])
        assert int(rec["count_neg_O"]) == int(ref["count_neg_O"])
        for f in ("min", "max", "mean"):
            np.testing.assert_allclose(rec[f], ref[f], rtol=0, atol=TOL64)
        np.testing.assert_array_equal(rec["argmin"], ref["argmin"])
        np.testing.assert_array_equal(rec["argmax"], ref["argmax"])
        n = int(rec["top_count"])
        assert n == int(ref["top_count"])
        if n:
            np.testing.assert_array_equal(hi["id"][:n], rhi["id"][:n])
            np.testing.assert_array_equal(lo["id"][:n], rlo["id"][:n])
            np.testing.assert_allclose(hi["value"][:n], rhi["value"][:n], atol=TOL64)
            np.testing.assert_allclose(lo["value"][:n], rlo["value"][:n], atol=TOL64)


def test_noalloc_rejects_sizes_beyond_limits():
    lib = P.load()
    S = torch.eye(8, dtype=torch.float64, device="cuda")
    rec = torch.zeros(240, dtype=torch.uint8, device="cuda")
    top = torch.zeros(2 * 32 * 16, dtype=torch.uint8, device="cuda")
    st = lib.thoi_order_record_noalloc(ctypes.c_void_p(S.data_ptr()), 8, 3, 17,
                                       ctypes.c_void_p(rec.data_ptr()),
                                       ctypes.c_void_p(top.data_ptr()), None)
    assert st == 3  # THOI_ERR_TOO_LARGE: top_m above 16
    st = lib.thoi_order_record_noalloc(ctypes.c_void_p(S.data_ptr()), 65, 3, 0,
                                       ctypes.c_void_p(rec.data_ptr()), None, None)
    assert st == 3  # N above 64


def test_noalloc_status_after_the_device_work():
    # errors found on the device come back as statuses: a zero variance is
    # an invalid argument; two identical variables make the pair singular
    S = np.eye(6)
    S[2, 2] = 0.0
    with pytest.raises(P.ThoiError) as e:
        P.thoi_order_record_noalloc(torch.as_tensor(S, device="cuda"), 3)
    assert e.value.code == 1  # THOI_ERR_INVALID_ARG
    S = workloads.random_corr(np.random.default_rng(81), 6)
    S[:, 4] = S[:, 1]
    S[4, :] = S[1, :]
    S[4, 4] = S[1, 1]
    with pytest.raises(P.ThoiError) as e:
        P.thoi_order_record_noalloc(torch.as_tensor(S, device="cuda"), 2)
    assert e.value.code == 4  # THOI_ERR_NOT_PD
    # and the next valid call is unaffected by the failed ones
    X, _ = workloads.small()
    S = oracle.copula_cov(X)
    ref, _, _ = _regular(S, 4, 0)
    rec, _, _ = P.thoi_order_record_noalloc(torch.as_tensor(S, device="cuda"), 4)
    np.testing.assert_allclose(rec["mean"], ref["mean"], rtol=0, atol=TOL64)


def test_noalloc_rejects_short_or_foreign_buffers():
    S = torch.eye(8, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        P.thoi_order_record_noalloc(S, 3, 4, rec_out=torch.zeros(239, dtype=torch.uint8,
                                                                 device="cuda"))
    with pytest.raises(ValueError):
        P.thoi_order_record_noalloc(S, 3, 4, top_out=torch.zeros(2 * 4 * 16 - 1,
                                                                 dtype=torch.uint8,
                                                                 device="cuda"))
    with pytest.raises(ValueError):
        P.thoi_order_record_noalloc(S, 3, 0, rec_out=torch.zeros(240, dtype=torch.uint8))


@pytest.mark.skipif(not torch.cuda.is_available() or torch.cuda.device_count() < 2,
                    reason="needs two GPUs")
def test_noalloc_rejects_memory_of_another_device():
    # the library runs on the current device: a covariance on another GPU is
    # an invalid argument, checked before any device work
    lib = P.load()
    S = torch.eye(8, dtype=torch.float64, device="cuda:1")
    rec = torch.zeros(240, dtype=torch.uint8, device="cuda:0")
    with torch.cuda.device(0):
        st = lib.thoi_order_record_noalloc(ctypes.c_void_p(S.data_ptr()), 8, 3, 0,
                                           ctypes.c_void_p(rec.data_ptr()), None, None)
    assert st == 1
