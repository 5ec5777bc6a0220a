"""Row sharding across ranks (one process per GPU): the row ranges, the
final pair exchange and the max-over-ranks timing, as world_size-2 gloo
process groups on the CPU.  The per-rank comparison is the CPU oracle, so
the test checks the sharding and exchange logic: the gathered result must
equal a one-rank run of the whole collection exactly."""
import os
import socket
import tempfile

import numpy as np
import pytest

from oracle import oracle_c as oc
from paper_1805_11254_gb300 import hoph, shard, synth

D, K, KG, AB, T, EPS = 1 << 16, 128, 32, (1, 1), (7, 10), 1e-4


@pytest.mark.parametrize("n", [0, 1, 2, 5, 10, 1000003])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_row_ranges_cover_contiguously(n, world):
    ranges = [shard.row_range(n, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        assert a1 == b0
    sizes = [r1 - r0 for r0, r1 in ranges]
    assert min(sizes) >= 0 and max(sizes) - min(sizes) <= 1


def test_row_range_rejects_bad_requests():
    for args in ((10, 2, 2), (10, -1, 2), (10, 0, 0), (-1, 0, 1)):
        with pytest.raises(ValueError):
            shard.row_range(*args)


def test_merge_restores_query_row_order():
    a = np.zeros(3, dtype=hoph.PAIR_DTYPE)
    a["query"], a["row"] = [0, 2, 5], [7, 1, 3]
    b = np.zeros(2, dtype=hoph.PAIR_DTYPE)
    b["query"], b["row"] = [0, 2], [2, 0]
    m = shard.merge_pairs([shard.globalize(a, 10), b])
    assert list(zip(m["query"], m["row"])) == [(0, 2), (0, 17), (2, 0), (2, 11), (5, 13)]
    assert len(shard.merge_pairs([])) == 0


def _oracle_pairs(q_rows, c_rows, z):
    acc = oc.query("hoph", q_rows, c_rows, KG, T[0], T[1], EPS, z=z, threads=1)["accepted"]
    out = np.zeros(len(acc), dtype=hoph.PAIR_DTYPE)
    out["query"], out["row"], out["groups"], out["matches"] = acc[:, 0], acc[:, 1], acc[:, 2], \
        acc[:, 3]
    return out


def _workload():
    w = synth.small_parity_workload(n=1201, n_queries=24)
    lo = oc.layout(D, K, KG, *AB)
    perm = oc.permutation(D, 1)
    c_rows = oc.sketch(w["ids"], w["off"], lo, perm=perm, threads=1)
    q_rows = oc.sketch(w["q_ids"], w["q_off"], lo, perm=perm, threads=1)
    z = np.asarray([int(lo[(g + 1) * KG] - lo[g * KG]) for g in range(K // KG)], dtype=np.uint64)
    return q_rows, c_rows, z


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        q_rows, c_rows, z = _workload()
        n = len(c_rows)

        def local_query(r0, r1):  # this rank holds rows [r0, r1) only
            return _oracle_pairs(q_rows, c_rows[r0:r1], z)

        everyone = shard.sharded_query(local_query, n)
        at_root = shard.sharded_query(local_query, n, dst=0)
        slowest = shard.max_over_ranks(1.5 + rank)
        np.save(os.path.join(out_dir, "all_%d.npy" % rank), everyone)
        if rank == 0:
            np.save(os.path.join(out_dir, "root.npy"), at_root)
        else:
            assert at_root is None
        with open(os.path.join(out_dir, "max_%d.txt" % rank), "w") as f:
            f.write(repr(slowest))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("n,batch,parts", [(1201, 100, 2), (1201, 100, 3), (10, 4, 5),
                                            (2, 1536, 2), (1, 10, 2), (0, 10, 1)])
def test_self_join_blocks_cover_every_block_once(n, batch, parts):
    blocks = [shard.self_join_blocks(n, batch, p, parts) for p in range(parts)]
    flat = sorted(b for bl in blocks for b in bl)
    n_blocks = (n - 1 + batch - 1) // batch if n > 1 else 0
    assert flat == list(range(n_blocks))
    # pair comparisons per part (block b: its queries against the rows from b*batch on)
    work = [sum(min(batch, n - 1 - b * batch) * (n - b * batch) for b in bl) for bl in blocks]
    if n_blocks >= 2 * parts:
        assert max(work) <= 1.6 * min(work)


def test_self_join_split_rejects_bad_requests():
    for args in ((10, 0, 0, 1), (10, 4, 2, 2), (10, 4, -1, 2), (10, 4, 0, 0), (-1, 4, 0, 1)):
        with pytest.raises(ValueError):
            shard.self_join_blocks(*args)


def _self_join_rows():
    q_rows, c_rows, z = _workload()
    return np.concatenate([c_rows, q_rows]), z


def _self_join_pairs(rows, z, blocks, batch):
    """The oracle's accepted pairs i < j whose query row i lies in `blocks`."""
    allp = _oracle_pairs(rows, rows, z)
    keep = (allp["query"] < allp["row"]) & np.isin(allp["query"] // batch, blocks)
    return allp[keep]


def _self_join_rank_main(rank, world, port, out_dir, batch):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        rows, z = _self_join_rows()

        def local_self_join(part, parts):  # every rank holds the whole collection
            return _self_join_pairs(rows, z, shard.self_join_blocks(len(rows), batch, part,
                                                                    parts), batch)

        np.save(os.path.join(out_dir, "sj_%d.npy" % rank), shard.sharded_self_join(local_self_join))
        np.save(os.path.join(out_dir, "mine_%d.npy" % rank), local_self_join(rank, world))
    finally:
        dist.destroy_process_group()


def test_two_rank_sharded_self_join_equals_one_rank():
    """The self-join split by blocks over 2 gloo ranks (each holding the whole
    collection, the oracle standing in for the GPU): the gathered pairs equal
    the one-rank self-join's, and both ranks found some of them."""
    import torch.multiprocessing as mp
    world, batch = 2, 100
    with tempfile.TemporaryDirectory() as tmp:
        mp.spawn(_self_join_rank_main, args=(world, _free_port(), tmp, batch), nprocs=world,
                 join=True)
        rows, z = _self_join_rows()
        allp = _oracle_pairs(rows, rows, z)
        want = allp[allp["query"] < allp["row"]]
        assert len(want) > 0  # the planted near duplicates
        for r in range(world):
            assert np.array_equal(np.load(os.path.join(tmp, "sj_%d.npy" % r)), want)
            assert len(np.load(os.path.join(tmp, "mine_%d.npy" % r))) > 0


def test_two_rank_sharded_query_equals_one_rank():
    import torch.multiprocessing as mp
    world = 2
    with tempfile.TemporaryDirectory() as tmp:
        mp.spawn(_rank_main, args=(world, _free_port(), tmp), nprocs=world, join=True)
        q_rows, c_rows, z = _workload()
        want = _oracle_pairs(q_rows, c_rows, z)
        assert len(want) > 0  # the planted near duplicates
        for r in range(world):
            got = np.load(os.path.join(tmp, "all_%d.npy" % r))
            assert np.array_equal(got, want)
            with open(os.path.join(tmp, "max_%d.txt" % r)) as f:
                assert float(f.read()) == 1.5 + world - 1
        assert np.array_equal(np.load(os.path.join(tmp, "root.npy")), want)
        # the split really put accepted pairs on both ranks' rows
        r0, r1 = shard.row_range(len(c_rows), 1, world)
        assert ((want["row"] >= r0) & (want["row"] < r1)).any()
        assert (want["row"] < r0).any()
