"""Id-range sharding across processes (one GPU each in production), tested on
the CPU: the library's host partitioner splits a request, each rank reduces
its range (here with the oracle, standing in for its GPU), the records are
all-gathered over gloo and merged by the library's host merge, and the merge
must equal the single-rank reduction of the whole request."""
import math
import os
import socket

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
import paper_2501_03381_gb300 as P  # noqa: E402

from records_pack import assert_same, pack  # noqa: E402

TOP_M = 12


def _work3(k):
    return 2 * k ** 3 + 6 * k ** 2


def _case():
    rng = np.random.default_rng(77)
    S = workloads.random_corr(rng, 13)
    # a not positive definite variable pair makes some nplets fail everywhere
    S[11, :] = S[12, :]
    S[:, 11] = S[:, 12]
    S[11, 11] = 1.0
    return S, list(range(2, 14))


def _reduce(S, orders, a, b):
    vals, fl = oracle.measures(S, orders, a, b)
    ids = np.arange(a, b, dtype=np.uint64)
    return pack(oracle.reduce_per_order(S.shape[0], orders, vals, ids, fl, top_m=TOP_M), TOP_M)


def _group_case():
    # four subjects x two conditions, one rank-deficient dataset
    rng = np.random.default_rng(78)
    Ss = [workloads.random_corr(rng, 11) for _ in range(8)]
    Ss[5][9, :] = Ss[5][10, :]
    Ss[5][:, 9] = Ss[5][:, 10]
    Ss[5][9, 9] = 1.0
    return Ss, list(range(3, 12))


def _reduce_group(Ss, orders, a, b, objective="cohen_d"):
    """Records of a group objective over ids [a, b), as the library lays them
    out: every measure slot carries the objective."""
    g, bad = oracle.group_measures(Ss, orders, "O", objective, a, b)
    ids = np.arange(a, b, dtype=np.uint64)
    recs = oracle.reduce_per_order(Ss[0].shape[0], orders, np.tile(g, (5, 1)), ids, bad,
                                   top_m=TOP_M)
    return pack(recs, TOP_M)


# ------------------------------------------------------------------ partition
@pytest.mark.parametrize("N,orders,R", [(13, list(range(2, 14)), 2), (10, [3, 10, 5], 7),
                                        (30, list(range(3, 31)), 8), (64, [32, 1, 2], 5),
                                        (5, [5], 3), (12, [6], 1000)])
def test_partition_balances_work(N, orders, R):
    b = P.thoi_partition(N, orders, R).astype(object)
    counts = [math.comb(N, k) for k in orders]
    total = sum(counts)
    assert b[0] == 0 and b[-1] == total
    assert all(b[i] <= b[i + 1] for i in range(R))
    # cumulative work of the first x ids, from Python integers
    offs = np.cumsum([0] + counts).tolist()

    def cum(x):
        w = 0
        for o, k in enumerate(orders):
            n = min(max(x - offs[o], 0), counts[o])
            w += n * _work3(k)
        return w

    W = cum(total)
    wmax = max(_work3(k) for k in orders)
    for r in range(1, R):
        target = W * r // R
        # the boundary is the first id at which the cumulative work reaches the target
        assert cum(b[r]) >= target
        assert b[r] == 0 or cum(b[r] - 1) < target or cum(b[r]) - target < wmax


def test_partition_rejects_bad_arguments():
    with pytest.raises(P.ThoiError):
        P.thoi_partition(10, [11], 2)
    with pytest.raises(P.ThoiError):
        P.thoi_partition(10, [3], 0)


# ------------------------------------------------------------------ merge, one process
@pytest.mark.parametrize("R", [1, 3, 5])
def test_merge_of_ranges_equals_whole(R):
    S, orders = _case()
    b = [int(x) for x in P.thoi_partition(S.shape[0], orders, R)]
    whole = _reduce(S, orders, 0, b[-1])
    blocks = [_reduce(S, orders, b[r], b[r + 1]) for r in range(R)]
    merged = P.thoi_merge_records(blocks, len(orders), TOP_M)
    assert_same(merged, whole, len(orders), TOP_M)


@pytest.mark.parametrize("objective,R", [("cohen_d", 3), ("mean", 4)])
def test_group_records_merge_of_ranges_equals_whole(objective, R):
    # group objectives shard like the measures: by id ranges, merged once
    Ss, orders = _group_case()
    N = Ss[0].shape[0]
    b = [int(x) for x in P.thoi_partition(N, orders, R)]
    whole = _reduce_group(Ss, orders, 0, b[-1], objective)
    blocks = [_reduce_group(Ss, orders, b[r], b[r + 1], objective) for r in range(R)]
    merged = P.thoi_merge_records(blocks, len(orders), TOP_M)
    assert_same(merged, whole, len(orders), TOP_M)
    recs, _, _ = P.parse_records(merged, len(orders), TOP_M)
    assert sum(int(r["n_not_pd"]) for r in recs) > 0


def test_merge_rejects_mismatched_orders():
    S, orders = _case()
    a = _reduce(S, orders[:3], 0, 10)
    b = _reduce(S, orders[1:4], 0, 10)
    with pytest.raises(P.ThoiError):
        P.thoi_merge_records([a, b], 3, TOP_M)


# ------------------------------------------------------------------ gloo ranks
def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        S, orders = _case()
        b = [int(x) for x in P.thoi_partition(S.shape[0], orders, world)]
        mine = _reduce(S, orders, b[rank], b[rank + 1])
        got = [None] * world
        dist.all_gather_object(got, mine)
        merged = P.thoi_merge_records(got, len(orders), TOP_M)
        np.save(os.path.join(outdir, f"merged{rank}.npy"), merged)
        # a group objective over eight datasets, sharded the same way
        Ss, gorders = _group_case()
        gb = [int(x) for x in P.thoi_partition(Ss[0].shape[0], gorders, world)]
        gmine = _reduce_group(Ss, gorders, gb[rank], gb[rank + 1])
        ggot = [None] * world
        dist.all_gather_object(ggot, gmine)
        gmerged = P.thoi_merge_records(ggot, len(gorders), TOP_M)
        np.save(os.path.join(outdir, f"gmerged{rank}.npy"), gmerged)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_partition_and_merge(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    S, orders = _case()
    whole = _reduce(S, orders, 0, oracle.count(S.shape[0], orders))
    Ss, gorders = _group_case()
    gwhole = _reduce_group(Ss, gorders, 0, oracle.count(Ss[0].shape[0], gorders))
    for r in range(world):
        merged = np.load(tmp_path / f"merged{r}.npy")
        assert_same(merged, whole, len(orders), TOP_M)
        gmerged = np.load(tmp_path / f"gmerged{r}.npy")
        assert_same(gmerged, gwhole, len(gorders), TOP_M)
