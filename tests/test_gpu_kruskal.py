"""GPU parity of the randomized Kruskal sampler (appendix, tree samplers:
Kruskal's algorithm on random edge weights): trees, labels, counts, hashes
and clouds equal the oracle's bit for bit, on single graphs and on a batch
of uneven graphs."""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2311_00869_gb300 as P

    return P


def _check(P, sb, g, seed, t0, K):
    it = sb.sample_trees_kruskal(seed, t0, K, want_in_tree=True)
    counts, hashes = sb.frustration()
    ref = O.mst_sample(g, seed, t0, K, want_in_tree=True)
    assert np.array_equal(it.cpu().numpy(), ref["in_tree"])
    assert np.array_equal(counts.cpu().numpy(), ref["counts"])
    assert np.array_equal(hashes.cpu().numpy().view(np.uint64), ref["hashes"])
    assert np.array_equal(P.unpack_labels(sb.label(), K), ref["labels"])
    return ref


@pytest.mark.parametrize("K", [1, 63, 64, 130])
def test_kruskal_small_graphs_match_oracle(P, K):
    sb = P.SignedBal(0)
    try:
        for case in range(3):
            n, u, v, s = synth.random_connected(40 + 30 * case, 60 + 40 * case, seed=900 + case)
            g = O.clean_graph(n, u, v, s)
            sb.load_graph(n, u, v, s)
            _check(P, sb, g, seed=case, t0=5 * case, K=K)
    finally:
        sb.close()


def test_kruskal_passes_give_identical_trees(P):
    """Trees are grown a pass of words at a time; one word per pass (four
    passes of 64 trees) gives the same trees, labels, counts and hashes as a
    single pass, equal to the oracle's."""
    sb = P.SignedBal(0)
    try:
        n, u, v, s = synth.random_connected(300, 900, seed=77)
        g = O.clean_graph(n, u, v, s)
        sb.load_graph(n, u, v, s)
        sb.set_tuning(mst_words=1)
        _check(P, sb, g, seed=3, t0=11, K=256)
        one = (sb.label().clone(), [x.clone() for x in sb.frustration()])
        sb.set_tuning(mst_words=0)
        sb.sample_trees_kruskal(3, 11, 256)
        assert np.array_equal(sb.label().cpu().numpy(), one[0].cpu().numpy())
        for a, b in zip(sb.frustration(), one[1]):
            assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
    finally:
        sb.close()


def test_kruskal_config1_cloud_matches_oracle(P):
    """The 1,000-vertex, 5,000-edge Erdos-Renyi graph with 64 trees: the
    cloud built from Kruskal trees equals the oracle's cloud of those trees."""
    sb = P.SignedBal(0)
    try:
        n, u, v, s = synth.er_graph()
        g = O.clean_graph(n, u, v, s)
        sb.load_graph(n, u, v, s)
        sb.cloud_reset()
        ref = _check(P, sb, g, seed=3, t0=0, K=64)
        cl, fr = sb.cloud()
        rc = O.cloud(ref["labels"], ref["counts"], t0=0)
        assert fr == rc["S"].min()
        assert np.array_equal(cl["first_tree"], rc["first_tree"])
        assert np.array_equal(cl["count"], rc["count"])
        assert np.array_equal(cl["S"], rc["S"])
        assert np.array_equal(cl["hash"], rc["H"])
    finally:
        sb.close()


def test_kruskal_edge_cases(P):
    """A single vertex, a single edge, a path (every tree the same), and a
    balanced graph (S = 0 on every tree, one state)."""
    sb = P.SignedBal(0)
    try:
        for n, u, v, s in ((1, [], [], []), (2, [0], [1], [-1]), (6, [0, 1, 2, 3, 4], [1, 2, 3, 4, 5],
                                                                    [1, -1, -1, 1, -1])):
            u, v, s = (np.array(u, np.int32), np.array(v, np.int32), np.array(s, np.int8))
            g = O.clean_graph(n, u, v, s)
            sb.load_graph(n, u, v, s)
            ref = _check(P, sb, g, seed=1, t0=0, K=70)
            assert np.all(ref["counts"] == 0)
        n, u, v, s, side = synth.planted_balanced(50, 80, seed=77)
        g = O.clean_graph(n, u, v, s)
        sb.load_graph(n, u, v, s)
        ref = _check(P, sb, g, seed=2, t0=9, K=100)
        assert np.all(ref["counts"] == 0)
    finally:
        sb.close()


def test_kruskal_batch_matches_per_graph_oracle(P):
    rng = np.random.Generator(np.random.PCG64(11))
    graphs = []
    for _ in range(17):
        n = int(np.exp(rng.uniform(np.log(6), np.log(400))))
        graphs.append(synth.chung_lu(n, 6.0, 2.5, float(rng.uniform(0.05, 0.3)), seed=int(rng.integers(1 << 30))))
    graphs.append((3, np.array([], np.int32), np.array([], np.int32), np.array([], np.int8)))
    sb = P.SignedBal(0)
    try:
        nv, mv = sb.load_batch(graphs)
        refs = [O.clean_graph(*gr) for gr in graphs]
        K = 100
        it = sb.sample_trees_kruskal(4, 2, K, want_in_tree=True).cpu().numpy()
        counts, hashes = sb.batch_frustration()
        counts, hashes = counts.cpu().numpy(), hashes.cpu().numpy().view(np.uint64)
        labels = P.unpack_labels(sb.label(), K)
        off = np.concatenate([[0], np.cumsum(nv)])
        eoff = np.concatenate([[0], np.cumsum(mv)])
        for gi, r in enumerate(refs):
            ref = O.mst_sample(r, 4, 2, K, want_in_tree=True)
            assert np.array_equal(counts[gi], ref["counts"]), gi
            assert np.array_equal(hashes[gi], ref["hashes"]), gi
            assert np.array_equal(labels[:, off[gi]:off[gi + 1]], ref["labels"]), gi
            assert np.array_equal(it[:, eoff[gi]:eoff[gi + 1]], ref["in_tree"]), gi
    finally:
        sb.close()


def test_kruskal_argument_and_state_errors(P):
    """Out-of-order calls and out-of-range arguments come back as status
    codes; the largest K of one call is still exact."""
    ARG, STATE = -1, -10
    sb = P.SignedBal(0)
    try:
        with pytest.raises(P.SignedBalError) as e:
            sb.sample_trees_kruskal(0, 0, 8)
        assert e.value.code == STATE
        n, u, v, s = synth.random_connected(50, 80, seed=6)
        g = O.clean_graph(n, u, v, s)
        sb.load_graph(n, u, v, s)
        for K, t0 in ((0, 0), (4097, 0), (8, -1)):
            with pytest.raises(P.SignedBalError) as e:
                sb.sample_trees_kruskal(0, t0, K)
            assert e.value.code == ARG
        host = np.zeros((8, g.m), np.uint8)  # in_tree must be device memory
        with pytest.raises(P.SignedBalError) as e:
            sb._check(sb.lib.sb_sample_trees_kruskal(sb.h, 0, 0, 8, host.ctypes.data))
        assert e.value.code == ARG
        _check(P, sb, g, seed=1, t0=0, K=4096)
    finally:
        sb.close()
