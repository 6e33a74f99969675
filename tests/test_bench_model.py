"""CPU checks of the bench's algorithmic work counts: the FLOPs it divides by
the kernel time for the roofline.  The prefix-shared counts are checked
against a walk of the kernels' loop structure on small N (every (k-1)-prefix
with a last variable after it built once; every (k-2)-prefix with a middle
and a last variable after it built once, one stored step per middle index,
one final step per nplet; every (k-3)-prefix with three more variables after
it built once, one stored step per next index and per middle index, one final
step per nplet)."""
import itertools
import math

import pytest

import bench


def _walk_one_level(N, k):
    f = 0.0
    P = k - 1
    for pre in itertools.combinations(range(N), P):
        last = [b for b in range(pre[-1] + 1, N)] if P else list(range(N))
        if not last:
            continue
        f += sum(bench.prefix_level_flops(i) for i in range(P))
        f += len(last) * (bench.prefix_level_flops(P) + 2.0 * P)
    return f


def _walk_two_level(N, k):
    f = 0.0
    GP = k - 2
    for g in itertools.combinations(range(N), GP):
        m = g[-1] if GP else -1
        mids = [a for a in range(m + 1, N - 1)]
        if not mids:
            continue
        f += sum(bench.prefix_level_flops(i) for i in range(GP))
        for a in mids:
            f += bench.prefix_level_flops(GP)
            f += (N - 1 - a) * (bench.prefix_level_flops(k - 1) + 2.0 * (k - 1))
    return f


def _walk_three_level(N, k):
    f = 0.0
    HP = k - 3
    for h in itertools.combinations(range(N), HP):
        m = h[-1] if HP else -1
        firsts = [a for a in range(m + 1, N - 2)]
        if not firsts:
            continue
        f += sum(bench.prefix_level_flops(i) for i in range(HP))
        for a1 in firsts:
            f += bench.prefix_level_flops(HP)
            for a2 in range(a1 + 1, N - 1):
                f += bench.prefix_level_flops(k - 2)
                f += (N - 1 - a2) * (bench.prefix_level_flops(k - 1) + 2.0 * (k - 1))
    return f


def _walk_four_level(N, k):
    f = 0.0
    IP = k - 4
    for pre in itertools.combinations(range(N), IP):
        m = pre[-1] if IP else -1
        zeros = [a for a in range(m + 1, N - 3)]
        if not zeros:
            continue
        f += sum(bench.prefix_level_flops(i) for i in range(IP))
        for a0 in zeros:
            f += bench.prefix_level_flops(IP)
            for a1 in range(a0 + 1, N - 2):
                f += bench.prefix_level_flops(k - 3)
                for a2 in range(a1 + 1, N - 1):
                    f += bench.prefix_level_flops(k - 2)
                    f += (N - 1 - a2) * (bench.prefix_level_flops(k - 1) + 2.0 * (k - 1))
    return f


@pytest.mark.parametrize("N", [7, 9])
def test_prefix_counts_match_loop_walk(N):
    for k in range(3, N + 1):
        assert bench.prefix_order_flops(N, k) == pytest.approx(_walk_one_level(N, k), rel=1e-12)
        assert bench.prefix2_order_flops(N, k) == pytest.approx(_walk_two_level(N, k), rel=1e-12)
        # the paired variant does the same algorithmic work as the two-level kernel
        assert bench.order_flops(N, k, 3) == bench.order_flops(N, k, 2)
        if k >= 5:
            assert bench.order_flops(N, k, 4) == pytest.approx(_walk_three_level(N, k),
                                                               rel=1e-12)
        if k >= 6:
            assert bench.order_flops(N, k, 5) == pytest.approx(_walk_four_level(N, k),
                                                               rel=1e-12)
        assert bench.order_flops(N, k, 0) == math.comb(N, k) * bench.flops_model(k)


def test_dense_model_and_workload_totals():
    # F(k) = 2/3 k^3 + 2 k^2 and the N = 30 workload's nplet count
    assert bench.flops_model(3) == pytest.approx(18 + 18)
    assert bench.total_nplets() == 2 ** 30 - 1 - 30 - math.comb(30, 2)
    assert bench.total_flops() == pytest.approx(
        sum(math.comb(30, k) * bench.flops_model(k) for k in range(3, 31)))
    # the prefix-shared kernels do less work than the dense factorisation
    for k in range(5, 21):
        assert bench.prefix2_order_flops(30, k) < bench.prefix_order_flops(30, k) < \
            math.comb(30, k) * bench.flops_model(k)


def test_traffic_figure_for_every_kernel_family():
    # every launch shape the autotuner can store maps to a kernel family with
    # a captured DRAM figure, and every figure is far below the 12 B of basis
    # values per nplet that the stored records path wrote
    shapes = [(1, 8, 0), (2, 8, 0), (4, 8, 0)] + [(1, c, p) for p in range(1, 6) for c in (1, 2)]
    fams = {bench.kernel_family(s) for s in shapes}
    assert fams == set(bench.TRAFFIC_BYTES_PER_NPLET)
    for fam, b in bench.TRAFFIC_BYTES_PER_NPLET.items():
        assert b is None or 0.0 < b < 0.01, fam
