"""CPU checks of the CUDA library: it loads, exports every entry point the
header declares, and its host-side logic (counting, unranking, record sizes,
option defaults, argument validation) matches the oracle.  No compute call
touches a GPU here."""
import ctypes
import math

import numpy as np
import pytest

import oracle
import paper_2501_03381_gb300 as P


@pytest.fixture(scope="module")
def lib():
    return P.load()


def test_exports_every_header_symbol(lib):
    syms = P.header_symbols()
    assert len(syms) >= 17
    for s in syms:
        assert hasattr(lib, s), s


def test_count_matches_oracle(lib):
    for N in (2, 7, 20, 30, 40, 64):
        for orders in ([1], list(range(3, N + 1)), [N], [2, 5, 3]):
            orders = [k for k in orders if 1 <= k <= N]
            if not orders:
                continue
            assert P.thoi_count(N, orders) == oracle.count(N, orders)


@pytest.mark.parametrize("N", [1, 5, 12])
def test_host_unrank_all_ids(N):
    orders = list(range(1, N + 1))
    walk = oracle.enumerate_subsets(N, orders)
    for gid, row in enumerate(walk):
        exp = [int(x) for x in row if x >= 0]
        assert list(P.thoi_unrank(N, orders, gid)) == exp


@pytest.mark.parametrize("N", [30, 60])
def test_host_unrank_sampled(N):
    orders = list(range(3, N + 1)) if N == 30 else [3, 4, 5, 30]
    total = oracle.count(N, orders)
    rng = np.random.default_rng(N)
    ids = np.unique(np.concatenate([rng.integers(0, total, 500, dtype=np.uint64),
                                    [0, total - 1]])).astype(np.uint64)
    # first and last id of every order
    off = 0
    extra = []
    for k in orders:
        c = math.comb(N, k)
        extra += [off, off + c - 1]
        off += c
    ids = np.unique(np.concatenate([ids, np.array(extra, dtype=np.uint64)]))
    ref = oracle.unrank_ids(N, orders, ids)
    for gid, row in zip(ids, ref):
        assert list(P.thoi_unrank(N, orders, int(gid))) == [int(x) for x in row if x >= 0]


def test_unrank_rejects_out_of_range():
    with pytest.raises(P.ThoiError):
        P.thoi_unrank(10, [3], math.comb(10, 3))


def test_records_bytes():
    assert P.thoi_records_bytes(28, 256) == 28 * 240 + 28 * 2 * 256 * 16
    assert P.thoi_records_bytes(1, 0) == 240


def test_default_options(lib):
    o = P.thoi_options()
    lib.thoi_default_options(ctypes.byref(o))
    assert o.precision == 0 and o.top_m == 256 and abs(o.pivot_tau - 1e-2) < 1e-9
    assert o.trace_tau == 100.0 and o.bias_correct == 0 and o.sigma32_source == 1


def test_status_strings(lib):
    for code in range(10):
        assert lib.thoi_status_string(code)


def test_create_validation_without_gpu(lib):
    h = ctypes.c_void_p()
    X = np.zeros((10, 3))
    opt = P.make_options()
    # N above the limit and bad sizes are rejected before any device work
    assert lib.thoi_create(ctypes.byref(h), X.ctypes.data, 100, 65, 65, 1, ctypes.byref(opt),
                           None) == 3
    assert lib.thoi_create(ctypes.byref(h), X.ctypes.data, 3, 3, 3, 1, ctypes.byref(opt),
                           None) == 1
    assert lib.thoi_create(ctypes.byref(h), None, 10, 3, 3, 1, ctypes.byref(opt), None) == 1
    assert lib.thoi_create(ctypes.byref(h), X.ctypes.data, 10, 3, 2, 1, ctypes.byref(opt),
                           None) == 1
    assert lib.thoi_create(ctypes.byref(h), X.ctypes.data, 10, 3, 3, 7, ctypes.byref(opt),
                           None) == 1


def test_group_entry_points_validate_without_gpu(lib):
    # null or empty groups, too many datasets and null contexts are rejected
    # before any device work
    orders = (ctypes.c_int32 * 1)(3)
    st = P.thoi_stats()
    null3 = (ctypes.c_void_p * 3)(None, None, None)
    big = (ctypes.c_void_p * 1025)()
    for ctxs, D in ((None, 3), (null3, 0), (big, 1025), (null3, 3)):
        assert lib.thoi_group_measures(ctxs, D, orders, 1, 0, 2**64 - 1, 3, 0, 0, None, 0,
                                       ctypes.byref(st), None) == 1
        assert lib.thoi_group_greedy(ctxs, D, 3, 4, 8, 3, 0, 1, None, None, ctypes.byref(st),
                                     None) == 1
        assert lib.thoi_group_anneal(ctxs, D, 3, 4, 8, 10, 1.0, 0.9, 0, 3, 0, 1, 0, None, None,
                                     None, None, ctypes.byref(st), None) == 1


def test_search_and_measure_entry_points_validate_without_gpu(lib):
    # a null context is rejected before any device work by every entry point
    st = P.thoi_stats()
    orders = (ctypes.c_int32 * 1)(3)
    masks = np.zeros(8, dtype=np.uint64)
    vals = np.zeros(8)
    assert lib.thoi_greedy(None, 3, 4, 4, 3, 1, masks.ctypes.data, vals.ctypes.data,
                           ctypes.byref(st), None) == 1
    assert lib.thoi_anneal(None, 3, 4, 4, 10, 1.0, 0.9, 0, 3, 1, 0, masks.ctypes.data,
                           vals.ctypes.data, masks.ctypes.data, vals.ctypes.data,
                           ctypes.byref(st), None) == 1
    assert lib.thoi_measures(None, orders, 1, 0, 2**64 - 1, 0, None, 0, ctypes.byref(st),
                             None) == 1
    assert lib.thoi_measures_grad(None, orders, 1, 3, None, ctypes.byref(st), None) == 1
    assert lib.thoi_set_cancel(None, 1) == 1
    assert lib.thoi_n(None) == 0
