"""Greedy search on the device (FP64 evaluation, device selection) against
the oracle's greedy search."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
import paper_2501_03381_gb300 as P  # noqa: E402

pytestmark = pytest.mark.gpu


def _members(mask):
    m = int(mask)
    return tuple(i for i in range(64) if m >> i & 1)


def _compare(S, k0, k1, kappa, measure, maximize, **ctx_kw):
    ref = oracle.greedy(S, k0, k1, kappa, measure, maximize)
    with P.Context(Sigma=S, **ctx_kw) as c:
        masks, values = c.greedy(k0, k1, kappa, measure, maximize)
    for lvl, (sets, vals) in enumerate(ref):
        n = len(sets)
        got = [_members(x) for x in masks[lvl, :n]]
        assert got == sets, (k0 + lvl, got[:4], sets[:4])
        np.testing.assert_allclose(values[lvl, :n], vals, rtol=0, atol=1e-10)
        assert np.all(masks[lvl, n:] == 0) and np.all(np.isnan(values[lvl, n:]))


@pytest.mark.parametrize("measure,maximize", [("O", True), ("O", False), ("S", True),
                                              ("TC", False), ("H", False)])
def test_greedy_matches_oracle(measure, maximize):
    S = workloads.random_corr(np.random.default_rng(41), 14)
    _compare(S, 3, 10, 32, measure, maximize)


def test_greedy_wide_masks_and_fp32_context():
    # 64-bit masks (N = 40); the context's FP32 precision does not change the
    # FP64 evaluation of the search
    S = workloads.random_corr(np.random.default_rng(42), 40)
    _compare(S, 3, 6, 16, "O", False, precision="f32_fix64")


def test_greedy_edges():
    S = workloads.random_corr(np.random.default_rng(43), 6)
    # (O vanishes for every pair, so searches start at triplets: at k = 2 only
    # rounding noise would order the ties)
    _compare(S, 3, 6, 100, "O", True)   # kappa above every order's count
    _compare(S, 4, 4, 5, "S", False)    # one order only
    with P.Context(Sigma=S) as c:
        with pytest.raises(P.ThoiError):
            c.greedy(3, 7, 4)  # k1 > N
        with pytest.raises(P.ThoiError):
            c.greedy(3, 4, 0)


def test_greedy_planted_redundancy():
    # on the planted system, maximising O from triplets stays inside the
    # redundant block (variables 0..9 share a latent) up to order 8
    X, _ = workloads.planted30()
    S = oracle.copula_cov(X)
    ref = oracle.greedy(S, 3, 9, 8, "O", True)
    with P.Context(torch.as_tensor(X, device="cuda")) as c:
        masks, values = c.greedy(3, 9, 8, "O", True)
    for lvl, (sets, vals) in enumerate(ref):
        assert [_members(x) for x in masks[lvl]] == sets
        np.testing.assert_allclose(values[lvl], vals, rtol=0, atol=1e-10)
        if lvl + 3 <= 8:
            assert all(max(s) <= 9 for s in sets)


def test_greedy_all_ties_fall_back_to_streaming_reduction():
    # identity correlation: every candidate's O is exactly 0, so each order's
    # radix select gathers more tied entries than it may keep and the search
    # is repeated with the streaming reduction; ties go to the smallest rank
    S = np.eye(60)
    _compare(S, 3, 5, 256, "O", True)
