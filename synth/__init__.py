"""Seeded synthetic signed-graph generators shared by the oracle tests and the GPU path.

This module holds no part of the method's arithmetic (no tree rule, hash,
labelling, counting or loss): it only draws raw COO edge lists with +/-1
signs, and graphL starting points, from numpy's PCG64 generator.  The graphs
stand in for the SNAP / Konect / Amazon signed networks of the paper's
experiments (Sec. 5-6, Tables of dataset sizes), which are not available here:
R-MAT and Chung-Lu give their power-law degree shape, and the planted faction
structure plus iid sign noise gives their mostly-positive sign mix.

Every generator returns (n, src int32[m], dst int32[m], sign int8[m]) (the two-faction
R-MAT can add the planted factions).
"""
from __future__ import annotations

import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _unique_pairs_in_order(a, b):
    """Canonical (min, max) pairs without loops, deduplicated, first-seen order."""
    lo = np.minimum(a, b).astype(np.int64)
    hi = np.maximum(a, b).astype(np.int64)
    keep = lo != hi
    key = (lo[keep] << 32) | hi[keep]
    _, first = np.unique(key, return_index=True)
    first.sort()
    key = key[first]
    return (key >> 32).astype(np.int32), (key & 0xFFFFFFFF).astype(np.int32)


def _collect_unique(draw, m_target, batch, max_rounds=64, batch_more=None):
    """Call draw(k) -> (a, b) until m_target unique undirected pairs exist."""
    acc_a, acc_b = [], []
    for i in range(max_rounds):
        a, b = draw(batch if (i == 0 or batch_more is None) else batch_more)
        acc_a.append(a)
        acc_b.append(b)
        u, v = _unique_pairs_in_order(np.concatenate(acc_a), np.concatenate(acc_b))
        if u.shape[0] >= m_target:
            return u[:m_target], v[:m_target]
    return u, v


def er_graph(n=1000, m=5000, neg_frac=0.2, seed=1001):
    """Erdos-Renyi: m distinct uniform unordered pairs, iid negative signs."""
    rng = _rng(seed)
    u, v = _collect_unique(lambda k: (rng.integers(0, n, k), rng.integers(0, n, k)), m, int(m * 1.2) + 16)
    sign = np.where(rng.random(u.shape[0]) < neg_frac, -1, 1).astype(np.int8)
    return n, u, v, sign


def rmat_edges(scale, m_target, abcd=(0.57, 0.19, 0.19, 0.05), seed=1002):
    """R-MAT recursive quadrant choice until m_target distinct undirected
    non-loop pairs exist, then a seeded random vertex permutation."""
    rng = _rng(seed)
    a, b, c, _ = abcd
    n = 1 << scale

    # quadrant thresholds on a 32-bit uniform integer
    ta, tab, tabc = (int(round(x * 2**32)) for x in (a, a + b, a + b + c))

    def draw(k):
        row = np.zeros(k, np.int64)
        col = np.zeros(k, np.int64)
        for _lvl in range(scale):
            r = rng.integers(0, 1 << 32, k, dtype=np.uint64)
            down = r >= tab
            right = ((r >= ta) & (r < tab)) | (r >= tabc)
            row <<= 1
            row |= down
            col <<= 1
            col |= right
        return row, col

    u, v = _collect_unique(draw, m_target, max(1024, int(m_target * 1.12)), batch_more=max(1024, m_target // 16))
    perm = rng.permutation(n).astype(np.int32)
    return n, perm[u], perm[v], rng


def rmat_two_faction(scale=20, m_target=1 << 24, noise=0.10, seed=1002, with_factions=False):
    """Planted two-faction balance (faction iid 50/50, sign = product of the
    faction signs) followed by iid sign flips with probability `noise`.
    with_factions=True also returns the planted faction (+1 / -1) of every
    vertex."""
    n, u, v, rng = rmat_edges(scale, m_target, seed=seed)
    fac = np.where(rng.random(n) < 0.5, 1, -1).astype(np.int8)
    sign = (fac[u] * fac[v]).astype(np.int8)
    flip = rng.random(u.shape[0]) < noise
    sign[flip] = -sign[flip]
    return (n, u, v, sign, fac) if with_factions else (n, u, v, sign)


RMAT_CHUNK = 1 << 22


def _rmat_chunk_keys(a):
    """One chunk of R-MAT draws as canonical pair keys (lo << 32 | hi), loops
    dropped, duplicates inside the chunk dropped (first-seen order kept)."""
    scale, k, abcd, seed, idx = a
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed, spawn_key=(idx,))))
    ta, tab, tabc = (int(round(x * 2**32)) for x in (abcd[0], abcd[0] + abcd[1], abcd[0] + abcd[1] + abcd[2]))
    row = np.zeros(k, np.int64)
    col = np.zeros(k, np.int64)
    for _lvl in range(scale):
        r = rng.integers(0, 1 << 32, k, dtype=np.uint64)
        row <<= 1
        row |= r >= tab
        col <<= 1
        col |= ((r >= ta) & (r < tab)) | (r >= tabc)
    lo, hi = np.minimum(row, col), np.maximum(row, col)
    key = ((lo << 32) | hi)[lo != hi]
    _, first = np.unique(key, return_index=True)
    first.sort()
    return key[first]


def rmat_edges_chunked(scale, m_target, abcd=(0.57, 0.19, 0.19, 0.05), seed=1003, workers=0):
    """R-MAT drawn in fixed chunks of RMAT_CHUNK pairs, chunk i from its own
    PCG64 stream (SeedSequence(seed, spawn_key=(i,))); the first m_target
    distinct pairs in chunk order are kept, then a seeded vertex permutation.
    The graph does not depend on `workers` (a spawned process pool)."""
    n = 1 << scale
    keys, have, nxt = [], 0, 0
    while True:
        nch = max(1, -(-int((m_target - have) * 1.15) // RMAT_CHUNK))
        tasks = [(scale, RMAT_CHUNK, abcd, seed, nxt + i) for i in range(nch)]
        nxt += nch
        if workers > 0:
            import concurrent.futures as cf
            import multiprocessing as mp

            with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
                keys.extend(ex.map(_rmat_chunk_keys, tasks))
        else:
            keys.extend(_rmat_chunk_keys(t) for t in tasks)
        allk = np.concatenate(keys)
        _, first = np.unique(allk, return_index=True)
        have = first.shape[0]
        if have >= m_target:
            first.sort()
            allk = allk[first[:m_target]]
            break
        keys = [allk[np.sort(first)]]
    rng = _rng(seed)
    perm = rng.permutation(n).astype(np.int32)
    return n, perm[(allk >> 32).astype(np.int64)], perm[(allk & 0xFFFFFFFF).astype(np.int64)], rng


def rmat_three_faction(scale=24, m_target=1 << 27, noise=0.15, probs=(0.948, 0.026, 0.026), seed=1003, workers=0):
    """Three factions (iid with `probs`), inter-faction edges negative,
    intra-faction positive, then iid flips with probability `noise`.  Edges
    come from the chunked R-MAT draw (`workers` only changes the speed)."""
    n, u, v, rng = rmat_edges_chunked(scale, m_target, seed=seed, workers=workers)
    fac = rng.choice(len(probs), size=n, p=np.asarray(probs) / np.sum(probs)).astype(np.int8)
    sign = np.where(fac[u] == fac[v], 1, -1).astype(np.int8)
    flip = rng.random(u.shape[0]) < noise
    sign[flip] = -sign[flip]
    return n, u, v, sign


def chung_lu(n, mean_deg=8.0, gamma=2.5, neg_frac=0.2, seed=1005, i0=1.0):
    """Chung-Lu: weights w_i ~ (i + i0)^(-1/(gamma-1)); m = n*mean_deg/2
    distinct pairs drawn by endpoint sampling proportional to w."""
    rng = _rng(seed)
    w = (np.arange(n, dtype=np.float64) + i0) ** (-1.0 / (gamma - 1.0))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    m_target = int(round(n * mean_deg / 2))

    def draw(k):
        return (np.minimum(np.searchsorted(cdf, rng.random(k)), n - 1),
                np.minimum(np.searchsorted(cdf, rng.random(k)), n - 1))

    u, v = _collect_unique(draw, m_target, int(m_target * 1.3) + 16, max_rounds=16)
    perm = rng.permutation(n).astype(np.int32)
    sign = np.where(rng.random(u.shape[0]) < neg_frac, -1, 1).astype(np.int8)
    return n, perm[u], perm[v], sign


def _chung_lu_args(a):
    return chung_lu(*a)


def uneven_batch(count=4096, n_lo=50, n_hi=50000, seed=1005, workers=0, select=None):
    """`count` Chung-Lu graphs, vertex counts log-uniform in [n_lo, n_hi],
    mean degree 8, exponent 2.5, negative fraction U(0.05, 0.30) per graph.
    workers > 0 draws them in a spawned process pool (same graphs).
    select (indices into the `count` graphs) yields only those graphs, each
    exactly as the full draw gives it."""
    rng = _rng(seed)
    ns = np.floor(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), count))).astype(np.int64)
    negs = rng.uniform(0.05, 0.30, count)
    seeds = rng.integers(0, 2**62, count)
    idx = range(count) if select is None else [int(i) for i in select]
    args = [(int(ns[i]), 8.0, 2.5, float(negs[i]), int(seeds[i])) for i in idx]
    if workers > 0:
        import concurrent.futures as cf
        import multiprocessing as mp

        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            yield from ex.map(_chung_lu_args, args, chunksize=16)
        return
    for a in args:
        yield chung_lu(*a)


def random_connected(n, extra, neg_frac=0.3, seed=0):
    """Small connected graph: a random labelled tree plus `extra` random
    non-tree pairs; iid signs."""
    rng = _rng(seed)
    par = np.array([rng.integers(0, i) for i in range(1, n)], dtype=np.int64)
    a = np.concatenate([np.arange(1, n), rng.integers(0, n, 4 * extra + 8)])
    b = np.concatenate([par, rng.integers(0, n, 4 * extra + 8)])
    u, v = _unique_pairs_in_order(a, b)
    u, v = u[: n - 1 + extra], v[: n - 1 + extra]
    sign = np.where(rng.random(u.shape[0]) < neg_frac, -1, 1).astype(np.int8)
    return n, u, v, sign


def planted_balanced(n, extra, seed=0):
    """Connected graph whose signs come from a random vertex bipartition
    (balanced by Harary's theorem); also returns the bipartition."""
    n, u, v, _ = random_connected(n, extra, seed=seed)
    rng = _rng(seed + 7)
    side = rng.integers(0, 2, n).astype(np.int8)
    sign = np.where(side[u] == side[v], 1, -1).astype(np.int8)
    return n, u, v, sign, side


def gamma0(n, R, seed=0):
    """graphL starting point: U(-1, 1) on the 2^-23 grid (exact in float32)."""
    rng = _rng(seed)
    k = rng.integers(0, 1 << 24, size=(n, R), dtype=np.int64)
    return (k.astype(np.float64) * 2.0**-23 - 1.0).astype(np.float32)
