"""Multi-rank graphBpp on the host: tree ranges per rank and the merge of the
per-rank frustration clouds, run as world-size-2 gloo process groups on CPU
with the oracle standing in for each rank's device work (BFS trees and
Kruskal trees shard the same way: both are pure functions of the tree index)."""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch.multiprocessing as mp

import synth
from paper_2311_00869_gb300 import shard

SEED, K, STEPS = 20231101, 24, 3


def _graph(O):
    n, u, v, s = synth.er_graph(n=60, m=150, neg_frac=0.3, seed=77)
    return O.clean_graph(n, u, v, s)


def _sample(O, g, t0, count, sampler):
    if sampler == "kruskal":
        return O.mst_sample(g, SEED, t0, count)
    return O.sample(g, SEED, t0, count)


def _part(O, g, t0, count, sampler):
    smp = _sample(O, g, t0, count, sampler)
    cl = O.cloud(smp["labels"], smp["counts"], t0=t0)
    first = cl["first_tree"]
    labels = [np.packbits(smp["labels"][int(f) - t0]) for f in first]
    return {"hash": cl["H"], "S": cl["S"], "count": cl["count"], "first_tree": first, "labels": labels}


def _rank_main(rank, world, port, out_path, with_labels, sampler):
    import torch.distributed as dist

    import oracle as O

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = _graph(O)
        parts = []
        for step in range(STEPS):
            t0, cnt = shard.tree_range(rank, world, step, K)
            parts.append(_part(O, g, t0, cnt, sampler))
        local = shard.merge_clouds(parts)
        if not with_labels:
            local.pop("labels")
        merged = shard.gather_cloud(local)
        if rank == 0:
            np.savez(out_path, **{k: merged[k] for k in ("hash", "S", "count", "first_tree")})
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("with_labels,sampler", [(True, "bfs"), (False, "bfs"), (True, "kruskal")])
def test_two_rank_cloud_equals_single_process(oracle, with_labels, sampler):
    world = 2
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "merged.npz")
        mp.start_processes(_rank_main, args=(world, _free_port(), out, with_labels, sampler), nprocs=world,
                           join=True, start_method="spawn")
        got = dict(np.load(out))
    g = _graph(oracle)
    total = STEPS * world * K
    smp = _sample(oracle, g, 0, total, sampler)
    ref = oracle.cloud(smp["labels"], smp["counts"], t0=0)
    assert len(ref["H"]) > 3  # several distinct states, so the merge is exercised
    np.testing.assert_array_equal(got["hash"], ref["H"])
    np.testing.assert_array_equal(got["S"], ref["S"])
    np.testing.assert_array_equal(got["count"], ref["count"])
    np.testing.assert_array_equal(got["first_tree"], ref["first_tree"])
    assert int(got["count"].sum()) == total


def test_tree_ranges_partition_the_trees():
    world, steps, k = 3, 4, 5
    seen = []
    for step in range(steps):
        for r in range(world):
            t0, c = shard.tree_range(r, world, step, k)
            seen.extend(range(t0, t0 + c))
    assert sorted(seen) == list(range(world * steps * k))
    with pytest.raises(ValueError):
        shard.tree_range(3, 3, 0, 5)


def test_merge_keeps_label_distinct_states_apart():
    a = {"hash": np.array([5], np.uint64), "S": np.array([2]), "count": np.array([3]),
         "first_tree": np.array([7]), "labels": [np.array([1, 0], np.uint8)]}
    b = {"hash": np.array([5, 9], np.uint64), "S": np.array([2, 4]), "count": np.array([1, 2]),
         "first_tree": np.array([2, 4]), "labels": [np.array([1, 1], np.uint8), np.array([0, 0], np.uint8)]}
    m = shard.merge_clouds([a, b])
    assert m["first_tree"].tolist() == [2, 4, 7]
    assert m["hash"].tolist() == [5, 9, 5]
    assert m["count"].tolist() == [1, 2, 3]
    # same vector from two ranks: one state, counts added, earliest first tree
    b["labels"][0] = np.array([1, 0], np.uint8)
    m = shard.merge_clouds([a, b])
    assert m["first_tree"].tolist() == [2, 4] and m["count"].tolist() == [4, 2]


def test_merge_without_labels_reports_collision():
    a = {"hash": np.array([5], np.uint64), "S": np.array([2]), "count": np.array([3]), "first_tree": np.array([7])}
    b = {"hash": np.array([5], np.uint64), "S": np.array([3]), "count": np.array([1]), "first_tree": np.array([1])}
    with pytest.raises(ValueError, match="collision"):
        shard.merge_clouds([a, b])
