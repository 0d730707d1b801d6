"""GPU parity of the batch of uneven graphs (one disjoint union): every graph's
cleaning, trees, labels, counts, hashes and cloud equal what the oracle
gives for that graph alone."""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu


def _graphs(count, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(6), np.log(400))))
        out.append(synth.chung_lu(n, 6.0, 2.5, float(rng.uniform(0.05, 0.3)), seed=int(rng.integers(1 << 30))))
    # a balanced graph and an isolated-vertex graph (LCC of a single vertex)
    n, u, v, s, _ = synth.planted_balanced(30, 40, seed=5)
    out.append((n, u, v, s))
    out.append((3, np.array([], np.int32), np.array([], np.int32), np.array([], np.int8)))
    return out


@pytest.mark.parametrize("K", [64, 130])
def test_batch_matches_per_graph_oracle(K):
    import paper_2311_00869_gb300 as P

    graphs = _graphs(23, seed=K)
    sb = P.SignedBal(0)
    nv, mv = sb.load_batch(graphs)
    refs = [O.clean_graph(*g) for g in graphs]
    assert list(nv) == [r.n for r in refs] and list(mv) == [r.m for r in refs]
    # the union's edge list is the graphs' edge lists, shifted
    eu, ev, eneg = (t.cpu().numpy() for t in sb.graph_edges())
    off = np.concatenate([[0], np.cumsum(nv)])
    eoff = np.concatenate([[0], np.cumsum(mv)])
    for g, r in enumerate(refs):
        sl = slice(eoff[g], eoff[g + 1])
        assert np.array_equal(eu[sl] - off[g], r.eu) and np.array_equal(ev[sl] - off[g], r.ev)
        assert np.array_equal(eneg[sl], r.eneg)
    sb.sample_trees(7, 3, K)
    counts, hashes = sb.batch_frustration()
    counts, hashes = counts.cpu().numpy(), hashes.cpu().numpy().view(np.uint64)
    labels = P.unpack_labels(sb.label(), K)  # (K, n_total)
    cl = sb.batch_cloud()
    for g, r in enumerate(refs):
        ref = O.sample(r, 7, 3, K)
        assert np.array_equal(counts[g], ref["counts"]), g
        assert np.array_equal(hashes[g], ref["hashes"]), g
        assert np.array_equal(labels[:, off[g]:off[g + 1]], ref["labels"]), g
        rc = O.cloud(ref["labels"], ref["counts"], t0=3)
        assert cl["n_states"][g] == rc["S"].shape[0]
        assert cl["fr_min"][g] == ref["counts"].min()
        e = cl["entries"][g]
        assert np.array_equal(e["first_tree"], rc["first_tree"])
        assert np.array_equal(e["count"], rc["count"])
        assert np.array_equal(e["S"], rc["S"])
        assert np.array_equal(e["hash"], rc["H"])
    sb.close()


def test_batch_graphl_per_graph():
    """graphL on a batch: loss, discrete loss, gradient and descent of every
    graph equal the per-graph float64 oracle (renormalised per graph)."""
    import torch

    import paper_2311_00869_gb300 as P

    graphs = _graphs(9, seed=3)
    sb = P.SignedBal(0)
    nv, mv = sb.load_batch(graphs)
    refs = [O.clean_graph(*g) for g in graphs]
    off = np.concatenate([[0], np.cumsum(nv)])
    R = 8
    gam = synth.gamma0(int(off[-1]), R, seed=11)
    G0 = torch.from_numpy(gam).cuda()
    loss, F = sb.graphL_fwd(G0)  # G x R in a batch
    loss = loss.reshape(len(graphs), R).cpu().numpy()
    F = F.reshape(len(graphs), R).cpu().numpy()
    # adjoint with a different upstream weight for every (graph, column)
    gout = np.random.default_rng(5).uniform(0.5, 2.0, size=(len(graphs), R)).astype(np.float32)
    grad = sb.graphL_bwd(G0, torch.from_numpy(gout.reshape(-1)).cuda()).cpu().numpy()
    out, exps, F_trace, F_final = sb.graphL_descent(G0, 0.05, 60, renorm_log2=16, trace=True)
    exps = exps.reshape(len(graphs), R).cpu().numpy()
    F_final = F_final.reshape(len(graphs), R).cpu().numpy()
    out = out.cpu().numpy()
    for g, r in enumerate(refs):
        sl = slice(off[g], off[g + 1])
        L64, F64 = O.graphl_loss_f64(r, gam[sl].astype(np.float64))
        prod = np.abs(gam[sl][r.eu].astype(np.float64) * gam[sl][r.ev])
        assert np.array_equal(F[g], F64), g
        assert np.all(np.abs(loss[g] - L64) <= 1e-5 * (0.5 * (1.0 + prod)).sum(axis=0) + 1e-6), g
        g64 = O.graphl_grad_f64(r, gam[sl].astype(np.float64), gout[g].astype(np.float64))
        assert np.linalg.norm(grad[sl] - g64) <= 1e-5 * np.linalg.norm(g64) + 1e-6, g
        ref, rexps, _ = O.graphl_descent_f64(r, gam[sl], 0.05, 60, renorm_log2=16)
        got = out[sl].astype(np.float64) * np.exp2(exps[g].astype(np.float64))[None, :]
        want = ref * np.exp2(rexps.astype(np.float64))[None, :]
        scale = np.abs(want).max(axis=0) + 1e-300
        assert np.all(np.abs(got - want) <= 1e-3 * scale[None, :]), g
        oF, _ = O.graphl_round_f32(r, out[sl])
        assert np.array_equal(F_final[g], oF), g
    sb.close()


def test_batch_of_64_benchmark_graphs_matches_per_graph_oracle():
    """64 graphs of the benchmark's uneven batch (4096 Chung-Lu graphs with
    50 to 50,000 vertices; the same seeded choice of 64 that the benchmark's
    CPU baseline times), loaded as one disjoint union, 256 trees in every
    graph: each graph's counts, state hashes and cloud equal the oracle's for
    that graph alone (Algorithm 1).  The large graphs have split (hub) rows
    and many BFS levels, and the scorer flushes per graph."""
    from concurrent.futures import ThreadPoolExecutor
    import os

    import paper_2311_00869_gb300 as P

    idx = np.sort(np.random.default_rng(7).choice(4096, size=64, replace=False))
    graphs = list(synth.uneven_batch(count=4096, select=idx))
    K = 256
    sb = P.SignedBal(0)
    try:
        nv, mv = sb.load_batch(graphs)
        sb.sample_trees(0, 0, K)
        counts, hashes = sb.batch_frustration()
        counts, hashes = counts.cpu().numpy(), hashes.cpu().numpy().view(np.uint64)
        cl = sb.batch_cloud()
    finally:
        sb.close()
    assert int(nv.max()) > 20000  # the shapes the case is meant to cover

    def ref(gi):
        r = O.clean_graph(*graphs[gi])
        smp = O.sample(r, 0, 0, K)
        return r.n, r.m, smp["counts"], smp["hashes"], O.cloud(smp["labels"], smp["counts"])

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        refs = list(ex.map(ref, range(len(graphs))))
    for g, (rn, rm, rc, rh, rcl) in enumerate(refs):
        assert (nv[g], mv[g]) == (rn, rm), g
        assert np.array_equal(counts[g], rc), g
        assert np.array_equal(hashes[g], rh), g
        assert cl["n_states"][g] == rcl["S"].shape[0], g
        assert cl["fr_min"][g] == rc.min(), g
        e = cl["entries"][g]
        assert np.array_equal(e["first_tree"], rcl["first_tree"]), g
        assert np.array_equal(e["count"], rcl["count"]), g
        assert np.array_equal(e["S"], rcl["S"]), g
        assert np.array_equal(e["hash"], rcl["H"]), g


def test_batch_steps_captured_equal_uncaptured_and_oracle():
    """sb_batch_steps runs several graphBpp steps over a batch with no host
    synchronisation; with use_graph the step is captured into a CUDA graph
    and replayed (the device moves the tree range on).  Both forms give, per
    graph, the oracle's smallest S over all the steps' trees and the
    oracle's number of distinct states in the last step; the last step's
    counts and hashes are the context's batch.  A second call reuses the
    captured graph from another first tree.  A stalled barrier during the
    steps is reported by sync() as SB_ERR_TIMEOUT."""
    import torch

    import paper_2311_00869_gb300 as P

    graphs = _graphs(21, seed=9)
    sb = P.SignedBal(0)
    try:
        nv, mv = sb.load_batch(graphs)
        refs = [O.clean_graph(*g) for g in graphs]
        K, steps = 64, 4
        first = None
        for t0 in (100, 1000):
            out = {}
            for use_graph in (True, False):
                fr, ns = sb.batch_steps(3, t0, K, steps, use_graph=use_graph)
                sb.sync()
                counts, hashes = sb.batch_frustration()
                out[use_graph] = (fr.cpu().numpy(), ns.cpu().numpy(), counts.cpu().numpy(),
                                  hashes.cpu().numpy().view(np.uint64))
            for a, b in zip(out[True], out[False]):
                assert np.array_equal(a, b)
            fr, ns, counts, hashes = out[True]
            first = fr if first is None else first
            for g, r in enumerate(refs):
                ref = O.sample(r, 3, t0, K * steps)
                assert fr[g] == ref["counts"].min(), g
                last = slice((steps - 1) * K, steps * K)
                assert np.array_equal(counts[g], ref["counts"][last]), g
                assert np.array_equal(hashes[g], ref["hashes"][last]), g
                rc = O.cloud(ref["labels"][last], ref["counts"][last], t0=t0 + (steps - 1) * K)
                assert ns[g] == rc["S"].shape[0], g
        # a stalled barrier in the steps comes back from sync(), and the context recovers
        sb.set_tuning(wait_us=20000, stall_test=1)
        sb.batch_steps(3, 0, K, 2, use_graph=False)
        with pytest.raises(P.SignedBalError) as e:
            sb.sync()
        assert e.value.code == -12
        sb.set_tuning(wait_us=0)
        fr, _ = sb.batch_steps(3, 100, K, steps, use_graph=True)
        sb.sync()
        assert np.array_equal(fr.cpu().numpy(), first)
    finally:
        sb.close()
