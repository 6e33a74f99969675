"""Simulated annealing chains on the device against the oracle's chains,
draw for draw (same counter-based generator, same moves, FP64 energies)."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
import paper_2501_03381_gb300 as P  # noqa: E402

pytestmark = pytest.mark.gpu


def _sets(masks):
    return [tuple(i for i in range(64) if int(m) >> i & 1) for m in masks]


@pytest.mark.parametrize("klo,khi,measure,maximize", [(3, 10, "O", True), (3, 10, "O", False),
                                                      (6, 6, "S", True), (4, 9, "TC", False)])
def test_anneal_matches_oracle(klo, khi, measure, maximize):
    S = workloads.random_corr(np.random.default_rng(61), 14)
    chains, iters, T0, alpha, seed = 24, 80, 0.3, 0.96, 12345
    ref = oracle.anneal(S, klo, khi, chains, iters, T0, alpha, measure, maximize, seed)
    with P.Context(Sigma=S) as c:
        fm, fv, bm, bv = c.anneal(klo, khi, chains, iters, T0, alpha, measure, maximize, seed)
    assert _sets(fm) == ref[0]
    assert _sets(bm) == ref[2]
    np.testing.assert_allclose(fv, ref[1], rtol=0, atol=1e-10)
    np.testing.assert_allclose(bv, ref[3], rtol=0, atol=1e-10)


def test_anneal_wide_masks():
    S = workloads.random_corr(np.random.default_rng(62), 40)
    ref = oracle.anneal(S, 3, 12, 8, 40, 0.5, 0.9, "O", True, 77)
    with P.Context(Sigma=S) as c:
        fm, fv, bm, bv = c.anneal(3, 12, 8, 40, 0.5, 0.9, "O", True, 77)
    assert _sets(fm) == ref[0] and _sets(bm) == ref[2]
    np.testing.assert_allclose(bv, ref[3], rtol=0, atol=1e-10)


def test_anneal_arguments():
    S = workloads.random_corr(np.random.default_rng(63), 8)
    with P.Context(Sigma=S) as c:
        for bad in [(3, 9, 4, 10, 1.0, 0.9), (5, 4, 4, 10, 1.0, 0.9), (3, 5, 0, 10, 1.0, 0.9),
                    (3, 5, 4, 10, 0.0, 0.9)]:
            with pytest.raises(P.ThoiError):
                c.anneal(*bad)
        with pytest.raises(P.ThoiError):
            c.anneal(3, 5, 4, 10, 1.0, 0.9, patience=-1)


@pytest.mark.parametrize("chains", [16384, 3])
def test_anneal_thread_and_warp_kernels(chains):
    # 16384 chains or more run a thread per chain, fewer a warp per chain; the
    # first chains of each match the oracle's (chains are independent)
    S = workloads.random_corr(np.random.default_rng(64), 20)
    iters, T0, alpha, seed = 30, 0.4, 0.95, 2024
    klo, khi = (3, 20) if chains == 3 else (3, 12)
    ref = oracle.anneal(S, klo, khi, 3, iters, T0, alpha, "O", True, seed)
    with P.Context(Sigma=S) as c:
        fm, fv, bm, bv = c.anneal(klo, khi, chains, iters, T0, alpha, "O", True, seed)
    assert _sets(fm[:3]) == ref[0] and _sets(bm[:3]) == ref[2]
    np.testing.assert_allclose(fv[:3], ref[1], rtol=0, atol=1e-10)
    np.testing.assert_allclose(bv[:3], ref[3], rtol=0, atol=1e-10)
    if chains > 3:
        assert all(3 <= bin(int(m)).count("1") <= 12 for m in fm)


def test_anneal_warp_kernel_order_32():
    # the largest order the annealing takes: 32 members, one row per lane
    S = workloads.random_corr(np.random.default_rng(65), 36)
    ref = oracle.anneal(S, 28, 32, 4, 25, 0.2, 0.9, "S", False, 5)
    with P.Context(Sigma=S) as c:
        fm, fv, bm, bv = c.anneal(28, 32, 4, 25, 0.2, 0.9, "S", False, 5)
    assert _sets(fm) == ref[0] and _sets(bm) == ref[2]
    np.testing.assert_allclose(bv, ref[3], rtol=0, atol=1e-9)


@pytest.mark.parametrize("chains", [24, 16384])
def test_anneal_patience_matches_oracle(chains):
    # early stop after `patience` steps without a better set (the paper's
    # second termination criterion), on the warp and the thread kernels
    S = workloads.random_corr(np.random.default_rng(66), 16)
    iters, T0, alpha, seed, p = 120, 0.05, 0.97, 31, 6
    ref = oracle.anneal(S, 3, 9, 24, iters, T0, alpha, "O", True, seed, patience=p)
    full = oracle.anneal(S, 3, 9, 24, iters, T0, alpha, "O", True, seed)
    assert ref[0] != full[0]  # some chains stopped early and ended elsewhere
    with P.Context(Sigma=S) as c:
        fm, fv, bm, bv = c.anneal(3, 9, chains, iters, T0, alpha, "O", True, seed, patience=p)
    assert _sets(fm[:24]) == ref[0] and _sets(bm[:24]) == ref[2]
    np.testing.assert_allclose(fv[:24], ref[1], rtol=0, atol=1e-10)
    np.testing.assert_allclose(bv[:24], ref[3], rtol=0, atol=1e-10)
