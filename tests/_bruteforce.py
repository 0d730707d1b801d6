"""Exhaustive references for tiny graphs (n <= 20), written from the
definitions, independent of the oracle's tree method."""
import numpy as np


def _states(n):
    """All vertex bipartitions with vertex 0 fixed to side 0, as an
    (2^(n-1), n) uint8 matrix."""
    k = np.arange(1 << (n - 1), dtype=np.int64)
    bits = ((k[:, None] >> np.arange(n - 1)[None, :]) & 1).astype(np.uint8)
    return np.concatenate([np.zeros((k.shape[0], 1), np.uint8), bits], axis=1)


def exact_frustration(n, u, v, neg):
    """Frustration index (Def. in Sec. 2): the fewest edges whose sign must
    change for balance; by Harary's theorem (item 4) this is the minimum over
    vertex bipartitions of the edges that disagree with the bipartition."""
    X = _states(n)
    u = np.asarray(u); v = np.asarray(v); neg = np.asarray(neg, np.uint8)
    bad = (X[:, u] ^ X[:, v] ^ neg[None, :]).sum(axis=1)
    return int(bad.min()), int((bad == 0).sum())


def max_cut(n, u, v):
    """Maximum cut by enumeration, through the Laplacian quadratic form
    cut(s) = s^T L s / 4 for s in {-1, +1}^n."""
    Lap = np.zeros((n, n))
    for a, b in zip(u, v):
        Lap[a, a] += 1; Lap[b, b] += 1; Lap[a, b] -= 1; Lap[b, a] -= 1
    S = 1.0 - 2.0 * _states(n).astype(np.float64)
    cut = np.einsum("ki,ij,kj->k", S, Lap, S) / 4.0
    return int(round(cut.max()))
