"""Sharding of graphBpp trees over ranks (one process per GPU) and the merge of
their frustration clouds.

The trees of graphBpp are independent samples (Sec. 3, Algorithm 1): tree t of
seed s is a pure function of (graph, s, t).  Rank r of W therefore takes, at
step i, the tree range [(i*W + r)*K, (i*W + r + 1)*K) and grows it with no
exchange on the data path.  The only cross-rank step is the merge of the
per-rank clouds at the end of a job: states are keyed by their 64-bit state
hash, counts add up, and the first tree of a state is the minimum over ranks,
so the merged cloud equals the one a single process would have built over the
union of the ranges (entries in first-appearance order).

With label bits supplied the merge also compares every pair of entries that
share a hash bit for bit and keeps distinct states apart (as the per-device
cloud does); without them, equal hashes are taken as one state, and an entry
pair with equal hash but different frustration count is reported as a
collision (ValueError).
"""
from __future__ import annotations

import numpy as np


def tree_range(rank: int, world: int, step: int, K: int) -> tuple[int, int]:
    """First tree index and count of rank `rank`'s range at step `step`."""
    if not (0 <= rank < world) or K < 0 or step < 0:
        raise ValueError("bad shard arguments")
    return (step * world + rank) * K, K


def merge_clouds(parts):
    """Merges clouds given as dicts of arrays hash / S / count / first_tree
    (optionally `labels`: one row of packed label bits per entry).  Returns the
    merged dict in order of first appearance."""
    keys = ("hash", "S", "count", "first_tree")
    with_labels = all(p.get("labels") is not None for p in parts) and len(parts) > 0
    states = {}  # hash -> list of [first_tree, S, count, labels]
    for p in parts:
        n = len(p["hash"])
        for k in keys:
            if len(p[k]) != n:
                raise ValueError(f"cloud part has {len(p[k])} {k} entries for {n} hashes")
        for i in range(n):
            h = int(np.uint64(p["hash"][i]))
            lab = np.asarray(p["labels"][i]) if with_labels else None
            bucket = states.setdefault(h, [])
            for st in bucket:
                if with_labels:
                    if np.array_equal(st[3], lab):
                        break
                elif st[1] == int(p["S"][i]):
                    break
                else:
                    raise ValueError(f"state hash {h:#018x} carries two frustration counts: hash collision")
            else:
                st = [int(p["first_tree"][i]), int(p["S"][i]), 0, lab]
                bucket.append(st)
            if with_labels and st[1] != int(p["S"][i]):
                raise ValueError("equal label vectors with different frustration counts")
            st[0] = min(st[0], int(p["first_tree"][i]))
            st[2] += int(p["count"][i])
    flat = sorted(((st[0], h, st) for h, b in states.items() for st in b), key=lambda x: x[0])
    out = {
        "hash": np.array([h for _, h, _ in flat], dtype=np.uint64),
        "S": np.array([st[1] for _, _, st in flat], dtype=np.int32),
        "count": np.array([st[2] for _, _, st in flat], dtype=np.int64),
        "first_tree": np.array([st[0] for _, _, st in flat], dtype=np.int64),
    }
    if with_labels:
        out["labels"] = [st[3] for _, _, st in flat]
    return out


def gather_cloud(part, group=None):
    """Host-side all-gather of every rank's cloud (torch.distributed, any
    backend) followed by the merge; every rank returns the merged cloud."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, part, group=group)
    return merge_clouds(parts)
