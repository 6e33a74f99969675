"""Parity of the CUDA library with the FP64 oracle (GPU required).

Tolerances (stated by the method's precision contract):
  * ranks, nplet indices, counts: bit-exact;
  * FP64 path and FP64 re-factored nplets: 1e-10 nats absolute;
  * FP32 path: 1e-4 nats absolute for nplets whose correlation submatrix has
    condition number below 1e4 (the ones the FP32 path keeps);
  * covariance: 1e-12 (FP64 path), 1e-6 relative (tensor-core FP32 path).
"""
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


# ------------------------------------------------------------------ copula front end
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("where", ["device", "host"])
def test_ranks_bit_exact(dtype, where):
    rng = np.random.default_rng(1)
    X = rng.integers(-20, 21, size=(777, 9)).astype(dtype)  # heavy ties
    X[5, 0], X[6, 0] = -0.0, 0.0
    Xin = torch.as_tensor(X, device="cuda") if where == "device" else torch.as_tensor(X)
    with P.Context(Xin) as c:
        R = c.ranks()
    np.testing.assert_array_equal(R, oracle.rank(X.astype(np.float64)))


def test_covariance_matches_oracle():
    for X in (workloads.small()[0], workloads.planted30()[0], workloads.plain(60, 2000, 4)):
        S = oracle.copula_cov(X)
        with _ctx(X) as c:
            S64, S32 = c.cov()
        np.testing.assert_allclose(S64, S, rtol=0, atol=1e-12)
        np.testing.assert_array_equal(S32, S64.astype(np.float32))
        with _ctx(X, sigma32_source="tensorcore") as c:
            _, S32tc = c.cov()
        # split-BF16 tensor-core GEMM: FP32-level accuracy, no systematic bias
        d = np.sqrt(np.outer(np.diag(S), np.diag(S)))
        assert np.abs((S32tc - S) / d).max() < 4e-7


def test_nonfinite_input_rejected():
    X = np.random.default_rng(2).standard_normal((50, 4))
    X[7, 2] = np.nan
    with pytest.raises(P.ThoiError) as e:
        P.Context(torch.as_tensor(X, device="cuda"))
    assert e.value.name == "THOI_ERR_NONFINITE_INPUT"


def test_failed_allocation_returns_oom_and_device_stays_usable():
    # a re-factor list of 2^40 entries (8 TiB) cannot be allocated: cudaMalloc
    # refuses it at once and the call returns THOI_ERR_OOM with nothing
    # queued; the context still answers, and a context with an automatic
    # list then evaluates normally
    X, orders = workloads.small()
    S = oracle.copula_cov(X)
    ref, _ = oracle.measures(S, orders)
    with _ctx(X, flag_capacity=1 << 40) as c:
        with pytest.raises(P.ThoiError) as e:
            c.measures(orders)
        assert e.value.name == "THOI_ERR_OOM"
        S64, _ = c.cov()
        assert np.abs(S64 - S).max() < 1e-12
    with _ctx(X) as c:
        out, _ = c.measures(orders)
        assert np.abs(out.double().cpu().numpy() - ref).max() < TOL32


# ------------------------------------------------------------------ enumeration
@pytest.mark.parametrize("N", [1, 6, 13, 20])
def test_device_unrank_all_ids(N):
    orders = list(range(1, N + 1))
    ref = oracle.enumerate_subsets(N, orders)
    ids = np.arange(len(ref), dtype=np.int64)
    got = P.thoi_unrank_device(N, orders, ids).cpu().numpy()
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("N,orders", [(30, list(range(3, 31))), (60, [3, 4, 5]), (64, [32, 2])])
def test_device_unrank_sampled(N, orders):
    total = oracle.count(N, orders)
    rng = np.random.default_rng(N)
    ids = [0, total - 1]
    off = 0
    for k in orders:
        c = math.comb(N, k)
        ids += [off, off + c - 1]
        off += c
    ids = np.unique(np.concatenate([rng.integers(0, total, 20000, dtype=np.uint64),
                                    np.array(ids, dtype=np.uint64)]))
    ref = oracle.unrank_ids(N, orders, ids)
    got = P.thoi_unrank_device(N, orders, ids.astype(np.int64)).cpu().numpy()
    np.testing.assert_array_equal(got, ref)


# ------------------------------------------------------------------ per-nplet measures
def _refs(S, orders, a=0, b=None, T_bias=0):
    out, fl = oracle.measures(S, orders, a, b, T_bias=T_bias)
    return out, fl


def test_small_fp64_all_nplets():
    X, orders = workloads.small()
    S = oracle.copula_cov(X)
    ref, _ = _refs(S, orders)
    with _ctx(X, precision="f64") as c:
        out, st = c.measures(orders)
    got = out.cpu().numpy()
    assert got.dtype == np.float64 and got.shape == ref.shape
    np.testing.assert_allclose(got, ref, rtol=0, atol=TOL64)


def test_small_fp32_fix_all_nplets():
    X, orders = workloads.small()
    S = oracle.copula_cov(X)
    ref, _ = _refs(S, orders)
    with _ctx(X) as c:
        out, st = c.measures(orders)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=TOL32)


@pytest.mark.parametrize("sigma32", ["tensorcore", "from_f64"])
def test_fmri_like_fp32_fix_all_nplets(sigma32):
    X, orders = workloads.fmri_like()  # N=20, 1,048,365 nplets
    S = oracle.copula_cov(X)
    ref, _ = _refs(S, orders)
    with _ctx(X, out_f64=True, sigma32_source=sigma32) as c:
        out, st = c.measures(orders)
    got = out.cpu().numpy()
    err = np.abs(got - ref).max(axis=1)
    assert (err < TOL32).all(), err
    assert st.nplets == ref.shape[1]


def test_fmri_like_fp64_all_nplets():
    X, orders = workloads.fmri_like()
    S = oracle.copula_cov(X)
    ref, _ = _refs(S, orders)
    with _ctx(X, precision="f64") as c:
        out, _ = c.measures(orders)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=TOL64)


def test_refactored_nplets_reach_fp64_tolerance():
    # force every nplet through the FP64 re-factor (trace threshold below 1)
    X, orders = workloads.small()
    S = oracle.copula_cov(X)
    ref, _ = _refs(S, orders)
    with _ctx(X, out_f64=True, trace_tau=0.5) as c:
        out, st = c.measures(orders)
    assert st.n_refactored == ref.shape[1]
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=TOL64)


def test_ragged_subranges_cross_orders():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((12, 12))
    S = A @ A.T + 0.5 * np.eye(12)
    orders = [7, 3, 12, 1, 5]
    total = oracle.count(12, orders)
    with _ctx(Sigma=S, precision="f64") as c:
        for a, b in [(0, total), (5, 6), (17, 1000), (790, 793), (total - 3, total), (4, 4)]:
            ref, _ = _refs(S, orders, a, b)
            out, _ = c.measures(orders, a, b)
            np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=TOL64)


def test_planted30_sampled_ranges_fp32_and_fp64():
    X, orders = workloads.planted30()
    S = oracle.copula_cov(X)
    total = oracle.count(30, orders)
    rng = np.random.default_rng(4)
    starts = rng.integers(0, total - 4000, 6)
    with _ctx(X, out_f64=True) as c32, _ctx(X, precision="f64") as c64:
        for a in list(starts) + [0, total - 4000]:
            a = int(a)
            b = a + 4000
            ref, _ = _refs(S, orders, a, b)
            o32, _ = c32.measures(orders, a, b)
            o64, _ = c64.measures(orders, a, b)
            np.testing.assert_allclose(o64.cpu().numpy(), ref, rtol=0, atol=TOL64)
            np.testing.assert_allclose(o32.cpu().numpy(), ref, rtol=0, atol=TOL32)


def test_closed_forms_on_device():
    N = 9
    rho = 0.6
    S = np.full((N, N), rho) + (1 - rho) * np.eye(N)
    with _ctx(Sigma=S, precision="f64") as c:
        for k in range(2, N + 1):
            out, _ = c.measures([k], 0, 1)
            ld = (k - 1) * math.log(1 - rho) + math.log(1 + (k - 1) * rho)
            ldm = (k - 2) * math.log(1 - rho) + math.log(1 + (k - 2) * rho)
            tc, dtc = -0.5 * ld, 0.5 * (k * ldm - (k - 1) * ld)
            np.testing.assert_allclose(out.cpu().numpy()[1:, 0], [tc, dtc, tc - dtc, tc + dtc],
                                       atol=1e-12)
    with _ctx(Sigma=np.eye(6), precision="f64") as c:
        out, _ = c.measures(range(1, 7))
        o = out.cpu().numpy()
        assert np.abs(o[1:]).max() < 1e-13
        ks = np.array([len(r[r >= 0]) for r in oracle.enumerate_subsets(6, range(1, 7))])
        np.testing.assert_allclose(o[0], ks * 1.4189385332046727, atol=1e-13)


def test_bias_correction_matches_oracle():
    X, orders = workloads.small()
    S = oracle.copula_cov(X)
    ref, _ = _refs(S, orders, T_bias=X.shape[0])
    with _ctx(X, precision="f64", bias_correct=True) as c:
        out, _ = c.measures(orders)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=TOL64)


def test_not_positive_definite():
    S = np.eye(5)
    S[0, 1] = S[1, 0] = 1.0
    ref, fl = _refs(S, [3])
    for prec in ("f64", "f32_fix64"):
        with _ctx(Sigma=S, precision=prec, out_f64=True) as c:
            with pytest.raises(P.ThoiError) as e:
                c.measures([3])
            assert e.value.name == "THOI_ERR_NOT_PD"


# ------------------------------------------------------------------ reductions
def _check_records(recs, hi, lo, ref_recs, tol, S, orders, top_m, o_ref=None):
    """Per-order records against the oracle's reduction.  Values within tol;
    the reported ids must carry the reported extreme values (near-ties may
    pick a different but equally valid id)."""
    for s_, (r, e) in enumerate(zip(recs, ref_recs)):
        assert int(r["k"]) == e["k"]
        assert int(r["count"]) == e["count"] + e["n_not_pd"]
        if e["count"] == 0:
            continue
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
        h, l_ = hi[s_][:n], lo[s_][:n]
        np.testing.assert_allclose(h["value"], e["top_hi_val"][:n], atol=tol)
        np.testing.assert_allclose(l_["value"], e["top_lo_val"][:n], atol=tol)
        tv, _ = oracle.measures_ids(S, orders, np.concatenate([h["id"], l_["id"]]))
        np.testing.assert_allclose(tv[3], np.concatenate([h["value"], l_["value"]]), atol=tol)
        assert len(set(h["id"].tolist())) == n and len(set(l_["id"].tolist())) == n
        # O < 0 count: exact up to the nplets whose reference O lies within
        # tol of zero (o_ref: the reference O values of this order, if given)
        near0 = int((np.abs(o_ref[s_]) <= tol).sum()) if o_ref is not None else 0
        assert abs(int(r["count_neg_O"]) - e["neg_O"]) <= max(near0, e["count"] // 10 ** 5)


@pytest.mark.parametrize("prec,tol", [("f64", TOL64), ("f32_fix64", TOL32)])
def test_records_fmri_like(prec, tol):
    X, orders = workloads.fmri_like()
    S = oracle.copula_cov(X)
    vals, fl = _refs(S, orders)
    ids = np.arange(vals.shape[1], dtype=np.uint64)
    ref = oracle.reduce_per_order(20, orders, vals, ids, fl, top_m=256)
    with _ctx(X, precision=prec) as c:
        (recs, hi, lo), st = c.measures(orders, reduction="per_order")
    _check_records(recs, hi, lo, ref, tol, S, orders, 256)


def test_records_small_topm_edge_cases():
    X, orders = workloads.small()
    S = oracle.copula_cov(X)
    vals, fl = _refs(S, orders)
    ids = np.arange(vals.shape[1], dtype=np.uint64)
    for top_m in (0, 1, 7, 1024):
        ref = oracle.reduce_per_order(10, orders, vals, ids, fl, top_m=max(top_m, 1))
        with _ctx(X, precision="f64", top_m=top_m) as c:
            (recs, hi, lo), _ = c.measures(orders, reduction="per_order")
        for s, k in enumerate(orders):
            assert int(recs[s]["count"]) == math.comb(10, k)
            n = int(recs[s]["top_count"])
            assert n == min(top_m, math.comb(10, k))
            if n:
                np.testing.assert_array_equal(hi[s][:n]["id"], ref[s]["top_hi_id"][:n])
                np.testing.assert_array_equal(lo[s][:n]["id"], ref[s]["top_lo_id"][:n])


def test_records_on_subrange_and_host_buffer():
    X, orders = workloads.small()
    S = oracle.copula_cov(X)
    a, b = 100, 700
    vals, fl = _refs(S, orders, a, b)
    ids = np.arange(a, b, dtype=np.uint64)
    ref = oracle.reduce_per_order(10, orders, vals, ids, fl, top_m=16)
    with _ctx(X, precision="f64", top_m=16) as c:
        buf = np.zeros(P.thoi_records_bytes(len(orders), 16), dtype=np.uint8)
        (recs, hi, lo), _ = c.measures(orders, a, b, reduction="per_order", out=buf)
        dbuf = torch.zeros(buf.size, dtype=torch.uint8, device="cuda")
        (recs2, hi2, lo2), _ = c.measures(orders, a, b, reduction="per_order", out=dbuf)
    assert np.array_equal(recs, recs2) and np.array_equal(hi, hi2)
    for s in range(len(orders)):
        assert int(recs[s]["count"]) == ref[s]["count"]
        if ref[s]["count"]:
            np.testing.assert_array_equal(recs[s]["argmin"], ref[s]["argmin"])
            np.testing.assert_array_equal(recs[s]["argmax"], ref[s]["argmax"])


# ------------------------------------------------------------------ gradient
@pytest.mark.parametrize("measure", ["O", "S", "H", "TC", "DTC"])
def test_grad_small_vs_oracle(measure):
    rng = np.random.default_rng(5)
    A = rng.standard_normal((12, 12))
    S = A @ A.T + 1.0 * np.eye(12)
    orders = [3, 4, 5]
    G = oracle.grad(S, orders, measure)
    with _ctx(Sigma=S) as c:
        g, _ = c.grad(orders, measure)
    g = g.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(g, G, rtol=2e-4, atol=2e-4 * np.abs(G).max())


def test_grad_c4_vs_oracle_and_fd():
    X, orders = workloads.grad60()
    S = oracle.copula_cov(X)
    G = oracle.grad(S, orders, "O")
    with _ctx(X) as c:
        g, st = c.grad(orders, "O")
    g = g.cpu().numpy().astype(np.float64)
    scale = np.abs(G).max()
    assert np.abs(g - G).max() < 2e-4 * scale
    rng = np.random.default_rng(6)
    for _ in range(4):
        i, j = sorted(rng.integers(0, 60, 2))
        fd = oracle.fd_grad_entry(S, orders, "O", int(i), int(j), h=1e-6)
        an = g[i, j] if i == j else 2 * g[i, j]
        assert abs(fd - an) < 1e-3 * max(1.0, abs(fd))


def test_autograd_function():
    rng = np.random.default_rng(7)
    A = rng.standard_normal((8, 8))
    S = A @ A.T + np.eye(8)
    St = torch.tensor(S, device="cuda", requires_grad=True)
    L = P.MeasureSum.apply(St, [3, 4], "O")
    L.backward()
    G = oracle.grad(S, [3, 4], "O")
    np.testing.assert_allclose(St.grad.cpu().numpy(), G, rtol=2e-4, atol=2e-4 * np.abs(G).max())
    vals, fl = oracle.measures(S, [3, 4])
    assert abs(L.item() - vals[3].sum()) < 1e-3


# ------------------------------------------------------------------ batching
# ------------------------------------------------------------------ large orders
def _wellcond(N, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((N, N))
    S = A @ A.T + N * np.eye(N)
    d = np.sqrt(np.diag(S))
    return S / np.outer(d, d)


@pytest.mark.parametrize("N,orders", [(32, list(range(21, 33))), (40, [24, 25, 33, 36])])
def test_large_orders_lane_group_and_generic(N, orders):
    # orders 21..32 run on the lane-group kernels (2 or 4 lanes per nplet),
    # above 32 on the generic kernel; 32-bit and 64-bit masks
    S = _wellcond(N, 8)
    total = oracle.count(N, orders)
    rng = np.random.default_rng(9)
    offs = np.cumsum([0] + [math.comb(N, k) for k in orders])
    ranges = []
    for s_ in range(len(orders)):
        a0, b0 = int(offs[s_]), int(offs[s_ + 1])
        for _ in range(2):
            a = int(rng.integers(a0, max(a0 + 1, b0 - 700)))
            ranges.append((a, min(b0, a + 700)))
        ranges.append((max(a0, b0 - 300), b0))
    with _ctx(Sigma=S, out_f64=True) as c32, _ctx(Sigma=S, precision="f64") as c64:
        for a, b in ranges:
            ref, _ = _refs(S, orders, a, b)
            o32, _ = c32.measures(orders, a, b)
            np.testing.assert_allclose(o32.cpu().numpy(), ref, rtol=0, atol=TOL32)
            o64, _ = c64.measures(orders, a, b)
            np.testing.assert_allclose(o64.cpu().numpy(), ref, rtol=0, atol=TOL64)
    if N != 32:
        return
    # per-order records of two large orders (10.7M nplets) against the FP64 path
    rec_orders = [24, 27]
    with _ctx(Sigma=S, top_m=64) as c32, _ctx(Sigma=S, precision="f64", top_m=64) as c64:
        (r32, h32, l32), _ = c32.measures(rec_orders, reduction="per_order")
        (r64, h64, l64), _ = c64.measures(rec_orders, reduction="per_order")
    for s_ in range(2):
        assert int(r32[s_]["count"]) == int(r64[s_]["count"])
        np.testing.assert_allclose(r32[s_]["min"], r64[s_]["min"], atol=TOL32)
        np.testing.assert_allclose(r32[s_]["max"], r64[s_]["max"], atol=TOL32)
        np.testing.assert_allclose(r32[s_]["mean"], r64[s_]["mean"], atol=TOL32)
        np.testing.assert_allclose(h32[s_]["value"], h64[s_]["value"], atol=TOL32)
        np.testing.assert_allclose(l32[s_]["value"], l64[s_]["value"], atol=TOL32)


# ------------------------------------------------------------------ autotuner
def test_autotune_cache_and_parity(tmp_path):
    import json
    X, orders = workloads.planted30()
    S = oracle.copula_cov(X)
    path = str(tmp_path / "tune.json")
    with _ctx(X, out_f64=True) as c:
        P.thoi_autotune(c.h, 12, 14, path)
        ents = json.load(open(path))
        ks = sorted(e["k"] for e in ents)
        # the cache is process-wide: earlier tunings in this process are kept too
        assert {12, 13, 14} <= set(ks)
        # one shape per order for records reduced in place, one for per-nplet output
        uses = {(e["k"], e["out"]) for e in ents}
        assert {(k, u) for k in (12, 13, 14) for u in (0, 1)} <= uses
        for e in (e for e in ents if 12 <= e["k"] <= 14):
            if e.get("prefix", 0):
                assert e["lanes"] == 1 and e["chunk"] in (1, 2, 4)
            else:
                assert e["lanes"] in (1, 2) and e["chunk"] in (4, 8)
        # the tuned shapes compute the same measures
        total = oracle.count(30, orders)
        off = sum(math.comb(30, k) for k in range(3, 13))
        a, b = off + 1000, off + 6000
        ref, _ = _refs(S, orders, a, b)
        out, _ = c.measures(orders, a, b)
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=TOL32)
        # a second call reads the cache and measures nothing new
        P.thoi_autotune(c.h, 12, 14, path)
        assert json.load(open(path)) == ents


def _force_shape(h, k, wide, lanes, chunk, path, prefix=0):
    """Make the library use one launch shape for order k by loading it
    through the autotuner's cache file."""
    import json
    props = torch.cuda.get_device_properties(0)
    ent = {"gpu": props.name, "sms": props.multi_processor_count, "k": k, "wide": wide,
           "lanes": lanes, "chunk": chunk, "blocks_per_sm": 0, "prefix": prefix}
    with open(path, "w") as fh:
        fh.write("[\n" + json.dumps(ent) + "\n]\n")
    P.thoi_autotune(h, k, k, path)


@pytest.mark.parametrize("k", [14, 17, 20, 23])
def test_all_lane_shapes_agree(k, tmp_path):
    # every kernel variant the autotuner can pick gives the oracle's values
    X, orders = workloads.planted30()
    S = oracle.copula_cov(X)
    off = sum(math.comb(30, q) for q in orders if q < k)
    a, b = off + 777, off + 2777
    ref, _ = _refs(S, orders, a, b)
    with _ctx(X, out_f64=True) as c:
        for lanes in (1, 2, 4):
            for chunk in (1, 8):
                _force_shape(c.h, k, 0, lanes, chunk, str(tmp_path / "f.json"))
                out, _ = c.measures(orders, a, b)
                np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=TOL32)
        _force_shape(c.h, k, 0, 1 if k <= 20 else 2, 8, str(tmp_path / "f.json"))


# ------------------------------------------------------------------ id-range sharding
def test_virtual_ranks_partition_and_merge():
    # R "ranks" on one GPU: each reduces its id range of the fMRI-shaped
    # request, the host merge of their records equals the whole-range records
    from records_pack import assert_same
    X, orders = workloads.fmri_like()
    top_m = 64
    with _ctx(X, top_m=top_m) as c:
        # one kernel for every range (the prefix-shared kernel covers whole
        # orders only), so that the extremes compare bit for bit
        import tempfile
        with tempfile.TemporaryDirectory() as td:
            for k in orders:
                _force_shape(c.h, k, 0, 1, 8, f"{td}/d{k}.json", prefix=0)
        per = P.thoi_records_bytes(len(orders), top_m)
        def rec_bytes(a, b):
            out = np.zeros(per, dtype=np.uint8)
            P.thoi_measures(c.h, orders, a, b, kind=1, out=out, top_m=top_m)
            return out
        total = P.thoi_count(20, orders)
        whole = rec_bytes(0, total)
        for R in (2, 5):
            b = [int(x) for x in P.thoi_partition(20, orders, R)]
            blocks = [rec_bytes(b[r], b[r + 1]) for r in range(R)]
            merged = P.thoi_merge_records(blocks, len(orders), top_m)
            # extremes, ids and top lists are identical; the means differ by
            # the order of the compensated FP32 block sums only
            assert_same(merged, whole, len(orders), top_m, mean_atol=1e-7)


# ------------------------------------------------------------------ prefix-shared kernel
@pytest.mark.parametrize("variant,chunk", [(1, 1), (1, 3), (2, 1), (2, 3), (3, 1), (3, 2),
                                           (4, 1), (4, 3), (5, 1), (5, 2)])
def test_prefix_kernel_every_order_matches_oracle(variant, chunk, tmp_path):
    # the prefix-shared kernels (bordered steps over a shared (k-1)-prefix,
    # variant 1, or (k-2)-prefix, variant 2, the latter with the last variables
    # two at a time, variant 3, and over a shared (k-3)-prefix with one stored
    # step per next index, variant 4, and over a (k-4)-prefix with two such
    # steps, variant 5) on every order of the fMRI-shaped workload (odd and
    # even numbers of last variables), every nplet against the oracle
    X, orders = workloads.fmri_like()
    S = oracle.copula_cov(X)
    with _ctx(X, out_f64=True) as c:
        for k in orders:
            _force_shape(c.h, k, 0, 1, chunk, str(tmp_path / f"p{k}.json"), prefix=variant)
            ref, _ = _refs(S, [k])
            got, _ = c.measures([k])
            np.testing.assert_allclose(got.cpu().numpy(), ref, rtol=0, atol=TOL32)


def test_prefix_kernel_wide_masks_and_records(tmp_path):
    # 64-bit masks (N = 40) and the records path, on a random correlation
    # matrix whose O values are not crowded around zero
    S = workloads.random_corr(np.random.default_rng(12), 40)
    orders = [3, 4]
    with _ctx(Sigma=S, out_f64=True, top_m=16) as c:
        for k in orders:
            _force_shape(c.h, k, 1, 1, 2, str(tmp_path / f"w{k}.json"), prefix=k - 1)
        for k in orders:
            ref, _ = _refs(S, [k])
            got, _ = c.measures([k])
            np.testing.assert_allclose(got.cpu().numpy(), ref, rtol=0, atol=TOL32)
        vals, fl = _refs(S, orders)
        ids = np.arange(vals.shape[1], dtype=np.uint64)
        ref_recs = oracle.reduce_per_order(40, orders, vals, ids, fl, top_m=16)
        (recs, hi, lo), _ = c.measures(orders, reduction="per_order")
        n3 = math.comb(40, 3)
        _check_records(recs, hi, lo, ref_recs, TOL32, S, orders, 16,
                       o_ref=[vals[3, :n3], vals[3, n3:]])


# ------------------------------------------------------------------ one-call API
def test_module_level_measures_and_measure_sum():
    # P.measures: create, evaluate, free in one call (device tensor or host
    # array); P.measure_sum: the autograd function
    X, orders = workloads.small()
    S = oracle.copula_cov(X)
    ref, _ = _refs(S, orders)
    out, st = P.measures(torch.as_tensor(X, device="cuda"), orders, out_f64=True)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=TOL32)
    (recs, hi, lo), _ = P.measures(X, orders, reduction="per_order", top_m=8)
    assert int(recs["count"].sum()) == ref.shape[1]
    np.testing.assert_allclose(recs["min"][:, 3], [ref[3, o].min() for o in _order_slices(orders)],
                               rtol=0, atol=TOL32)
    rng = np.random.default_rng(81)
    A = rng.standard_normal((7, 7))
    Sg = A @ A.T + np.eye(7)
    St = torch.tensor(Sg, device="cuda", requires_grad=True)
    L = P.measure_sum(St, [3, 4], "S")
    L.backward()
    G = oracle.grad(Sg, [3, 4], "S")
    np.testing.assert_allclose(St.grad.cpu().numpy(), G, rtol=2e-4, atol=2e-4 * np.abs(G).max())


def _order_slices(orders, N=10):
    offs = np.cumsum([0] + [math.comb(N, k) for k in orders])
    return [slice(int(offs[i]), int(offs[i + 1])) for i in range(len(orders))]


def test_three_level_prefix_kernel_wide_masks(tmp_path):
    # the three-level kernel on 64-bit masks (N = 34), every nplet of order 5
    # against the oracle, and the records of orders 5 and 6 against those of
    # the dense kernel
    S = workloads.random_corr(np.random.default_rng(21), 34)
    with _ctx(Sigma=S, out_f64=True, top_m=16) as c:
        _force_shape(c.h, 5, 1, 1, 2, str(tmp_path / "t5.json"), prefix=4)
        ref, _ = _refs(S, [5])
        got, _ = c.measures([5])
        np.testing.assert_allclose(got.cpu().numpy(), ref, rtol=0, atol=TOL32)
        _force_shape(c.h, 6, 1, 1, 1, str(tmp_path / "t6.json"), prefix=4)
        (r3, h3, l3), _ = c.measures([5, 6], reduction="per_order")
        for k in (5, 6):
            _force_shape(c.h, k, 1, 1, 8, str(tmp_path / f"d{k}.json"), prefix=0)
        (r0, h0, l0), _ = c.measures([5, 6], reduction="per_order")
    for q in range(2):
        np.testing.assert_allclose(r3[q]["min"], r0[q]["min"], rtol=0, atol=TOL32)
        np.testing.assert_allclose(r3[q]["max"], r0[q]["max"], rtol=0, atol=TOL32)
        np.testing.assert_allclose(r3[q]["mean"], r0[q]["mean"], rtol=0, atol=1e-6)
        assert int(r3[q]["count"]) == int(r0[q]["count"])
        np.testing.assert_allclose(h3[q]["value"][:16], h0[q]["value"][:16], rtol=0, atol=TOL32)
        np.testing.assert_allclose(l3[q]["value"][:16], l0[q]["value"][:16], rtol=0, atol=TOL32)


@pytest.mark.parametrize("variant", [2, 3, 4, 5])
@pytest.mark.parametrize("N,orders", [(24, [21, 22]), (26, [23, 24])])
def test_prefix_kernels_orders_21_to_24(variant, N, orders, tmp_path):
    # the two-, three- and four-level kernels at the orders beyond the
    # one-level kernel's, every nplet against the oracle, per nplet and as
    # records
    S = workloads.random_corr(np.random.default_rng(33), N)
    with _ctx(Sigma=S, out_f64=True, top_m=8) as c:
        for k in orders:
            _force_shape(c.h, k, 0, 1, 1, str(tmp_path / f"q{k}.json"), prefix=variant)
        ref, fl = _refs(S, orders)
        got, _ = c.measures(orders)
        np.testing.assert_allclose(got.cpu().numpy(), ref, rtol=0, atol=TOL32)
        ids = np.arange(ref.shape[1], dtype=np.uint64)
        ref_recs = oracle.reduce_per_order(N, orders, ref, ids, fl, top_m=8)
        (recs, hi, lo), _ = c.measures(orders, reduction="per_order")
        for q, e in enumerate(ref_recs):
            np.testing.assert_allclose(recs[q]["min"], e["min"], atol=TOL32)
            np.testing.assert_allclose(recs[q]["max"], e["max"], atol=TOL32)
            np.testing.assert_allclose(recs[q]["mean"], e["mean"], atol=TOL32)
