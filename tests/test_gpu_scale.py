"""GPU parity at paper scale: the R-MAT graph with 2^24 vertex ids and 2^27
undirected edges (three factions, 15 % sign noise), 4096 trees in one
sample_trees call as the benchmark runs it.  The 128 trees [0, 64) and
[4032, 4096) (the first and the last word of 64 trees) are checked against
the oracle bit for bit: counts, state hashes and labels; the cloud must hold
every tree once and its minimum."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

K = 4096


@pytest.fixture(scope="module")
def graph():
    n, u, v, s = synth.rmat_three_faction(scale=24, m_target=1 << 27, workers=os.cpu_count() or 1)
    return n, u, v, s


@pytest.mark.timeout(1800)
def test_rmat_2pow24_sampled_trees(graph):
    import paper_2311_00869_gb300 as P

    n, u, v, s = graph
    sb = P.SignedBal(0)
    try:
        n1, m1, _ = sb.load_graph(n, u, v, s)
        sb.cloud_reset(max_states=K + 64)
        sb.sample_trees(0, 0, K)
        counts, hashes = sb.frustration()
        counts, hashes = counts.cpu().numpy(), hashes.cpu().numpy().view(np.uint64)
        labw = sb.label().cpu().numpy().view(np.uint64)
        cl, fr_min = sb.cloud()
    finally:
        sb.close()
    g = O.clean_graph(n, u, v, s)
    assert (n1, m1) == (g.n, g.m)

    trees = list(range(64)) + list(range(K - 64, K))
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        refs = list(ex.map(lambda t: O.sample(g, 0, t, 1), trees))
    W = K // 64
    first_last = np.ascontiguousarray(labw[:, [0, W - 1]])  # unpacking all 64 words would take 30 GB
    bits = np.unpackbits(first_last.view(np.uint8).reshape(labw.shape[0], -1), axis=1, bitorder="little")
    for t, ref in zip(trees, refs):
        assert counts[t] == ref["counts"][0], t
        assert hashes[t] == ref["hashes"][0], t
        col = t if t < 64 else 64 + (t - 64 * (W - 1))
        assert np.array_equal(bits[:, col], ref["labels"][0]), t
    assert np.all(counts >= 0) and np.all(counts <= g.m - g.n + 1)
    assert int(cl["count"].sum()) == K
    assert fr_min == int(counts.min())
    assert len(np.unique(cl["hash"])) == cl["hash"].shape[0]
