"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

graphBpp results are integers and must match bit for bit (trees, labels,
counts, hashes, cloud).  graphL runs in float32 against the oracle's float64
within the tolerances of the float32 reading (R12): loss within
1e-5 * sum_e (1 + |G_u G_v|) / 2, gradient within 1e-5 relative in norm.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2311_00869_gb300 as P

    return P


@pytest.fixture()
def sb(P):
    s = P.SignedBal(0)
    yield s
    s.close()


def load_both(sb, n, u, v, s, flags=O.LOAD_LCC | O.LOAD_MERGE_DUP):
    g = O.clean_graph(n, u, v, s, flags)
    n1, m1, vmap = sb.load_graph(n, u, v, s, flags, want_vmap=True)
    assert (n1, m1) == (g.n, g.m)
    assert np.array_equal(vmap, g.vmap)
    return g


def check_batch(P, sb, g, seed, t0, K, parents=False, labels=True):
    par = sb.sample_trees(seed, t0, K, want_parents=parents)
    counts, hashes = sb.frustration()
    ref = O.sample(g, seed, t0, K, want_labels=labels, want_parents=parents)
    assert np.array_equal(counts.cpu().numpy(), ref["counts"])
    assert np.array_equal(hashes.cpu().numpy().view(np.uint64), ref["hashes"])
    if parents:
        assert np.array_equal(par.cpu().numpy(), ref["parents"])
    if labels:
        lab = P.unpack_labels(sb.label(), K)
        assert np.array_equal(lab, ref["labels"])
    return ref


# ------------------------------------------------------------------ ingest

@pytest.mark.parametrize("case", range(4))
def test_ingest_matches_oracle(sb, case):
    rng = np.random.Generator(np.random.PCG64(50 + case))
    n = 300 + 200 * case
    m = 2 * n
    a = rng.integers(0, n, m)
    b = rng.integers(0, n, m)
    keep = a != b
    a, b = a[keep], b[keep]
    # repeat some pairs, reversed, with the same sign (merged duplicates)
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    key, idx = np.unique(lo * n + hi, return_index=True)
    a, b = a[idx], b[idx]
    s = np.where(rng.random(a.shape[0]) < 0.3, -1, 1).astype(np.int8)
    rep = rng.integers(0, a.shape[0], a.shape[0] // 5)
    a2 = np.concatenate([a, b[rep]]).astype(np.int32)
    b2 = np.concatenate([b, a[rep]]).astype(np.int32)
    s2 = np.concatenate([s, s[rep]]).astype(np.int8)
    g = load_both(sb, n, a2, b2, s2)
    u, v, neg = (t.cpu().numpy() for t in sb.graph_edges())
    assert np.array_equal(u, g.eu) and np.array_equal(v, g.ev) and np.array_equal(neg, g.eneg)
    rp, col, cneg = (t.cpu().numpy() for t in sb.graph_csr())
    assert np.array_equal(rp, g.rowptr.astype(np.int32))
    assert np.array_equal(col, g.col) and np.array_equal(cneg, g.colneg)


def test_ingest_from_device_and_pinned_host(sb):
    n, u, v, s = synth.er_graph(400, 1600, 0.3, seed=3)
    g = O.clean_graph(n, u, v, s)
    for conv in (lambda x: torch.from_numpy(x).cuda(), lambda x: torch.from_numpy(x).pin_memory()):
        n1, m1, _ = sb.load_graph(n, conv(u), conv(v), conv(s))
        assert (n1, m1) == (g.n, g.m)
        uu, vv, nn = (t.cpu().numpy() for t in sb.graph_edges())
        assert np.array_equal(uu, g.eu) and np.array_equal(vv, g.ev) and np.array_equal(nn, g.eneg)


def test_ingest_errors_match_oracle(P, sb):
    cases = [
        (3, [0, 1], [1, 1], [1, 1], 3),
        (3, [0, 1], [1, 2], [1, 0], 3),
        (3, [0, 1], [1, 3], [1, 1], 3),
        (3, [0, 1, 1], [1, 2, 0], [1, 1, -1], 3),
        (3, [0, 1, 1], [1, 2, 0], [1, 1, 1], O.LOAD_LCC),
        (4, [0, 2], [1, 3], [1, 1], O.LOAD_MERGE_DUP),
        (3, [0, 1, 1, 2], [2, 1, 0, 5], [7, 1, 1, 1], 3),  # first bad edge decides
    ]
    for n, a, b, s, flags in cases:
        a = np.array(a, np.int32)
        b = np.array(b, np.int32)
        s = np.array(s, np.int8)
        with pytest.raises(O.OracleError) as eo:
            O.clean_graph(n, a, b, s, flags)
        with pytest.raises(P.SignedBalError) as eg:
            sb.load_graph(n, a, b, s, flags)
        assert eg.value.code == eo.value.code


def test_single_vertex_and_single_edge(P, sb):
    g = load_both(sb, 5, np.array([], np.int32), np.array([], np.int32), np.array([], np.int8))
    assert g.n == 1 and g.m == 0
    check_batch(P, sb, g, 0, 0, 3, parents=True)
    g = load_both(sb, 2, np.array([1], np.int32), np.array([0], np.int32), np.array([-1], np.int8))
    check_batch(P, sb, g, 9, 5, 70, parents=True)


# ------------------------------------------------------------------ graphBpp

@pytest.mark.parametrize("K", [1, 63, 64, 130])
def test_trees_labels_counts_small(P, sb, K):
    n, u, v, s = synth.random_connected(60, 90, seed=K)
    g = load_both(sb, n, u, v, s)
    check_batch(P, sb, g, seed=K + 1, t0=7, K=K, parents=True)


def test_split_rows_hub(P, sb):
    # vertex 0 joins 2000 others (split into several chunks) plus a random mesh
    n, a, b, s = _hub_graph(seed=77, n=2001, extra=2600, neg=0.35)
    g = load_both(sb, n, a, b, s)
    assert np.diff(g.rowptr).max() > 1536
    check_batch(P, sb, g, seed=5, t0=0, K=200, parents=True)
    check_batch(P, sb, g, seed=6, t0=0, K=2048 + 33, parents=False)


def test_config1_plain_equals_batched_and_oracle(P, sb):
    n, u, v, s = synth.er_graph()
    g = load_both(sb, n, u, v, s)
    ref = check_batch(P, sb, g, seed=0, t0=0, K=64, parents=True)
    cl, fr = sb.cloud()
    rc = O.cloud(ref["labels"], ref["counts"])
    assert np.array_equal(cl["first_tree"], rc["first_tree"])
    assert np.array_equal(cl["count"], rc["count"])
    assert np.array_equal(cl["S"], rc["S"])
    assert np.array_equal(cl["hash"], rc["H"])
    assert fr == rc["S"].min()
    # plain path: one tree per call, cloud accumulated over 64 calls
    sb.cloud_reset()
    for t in range(64):
        sb.sample_trees(0, t, 1)
        c1, h1 = sb.frustration()
        assert c1.item() == ref["counts"][t]
        sb.cloud()
    cl2, fr2 = sb.cloud()
    for k in ("first_tree", "count", "S", "hash"):
        assert np.array_equal(cl2[k], cl[k])


def test_rmat_multiword_ragged(P, sb):
    n, u, v, s = synth.rmat_two_faction(scale=13, m_target=1 << 16, seed=12)
    g = load_both(sb, n, u, v, s)
    K = 32 * 64 + 52  # two BFS launches, ragged last word
    sb.sample_trees(11, 1000, K)
    counts, hashes = sb.frustration()
    ref = O.sample(g, 11, 1000, K, want_labels=True)
    assert np.array_equal(counts.cpu().numpy(), ref["counts"])
    assert np.array_equal(hashes.cpu().numpy().view(np.uint64), ref["hashes"])
    lab = P.unpack_labels(sb.label(), K)
    assert np.array_equal(lab, ref["labels"])


@pytest.mark.parametrize("words", [3, 8, 13, 32])
def test_bfs_words_per_launch_agree_with_the_oracle(P, sb, words):
    """Any number of 64-tree words per BFS launch gives the oracle's trees,
    labels, counts and hashes, with split rows, parents and a ragged last
    word (the words of a call split over launches of `words` words)."""
    n, a, b, s = _hub_graph(seed=91, n=1500, extra=4000, neg=0.3)
    g = load_both(sb, n, a, b, s)
    assert np.diff(g.rowptr).max() > 1024  # split rows
    sb.set_tuning(bfs_words=words)
    check_batch(P, sb, g, seed=17 + words, t0=300, K=64 * words - 5, parents=True)
    check_batch(P, sb, g, seed=18 + words, t0=7, K=64 * 64, parents=False)
    sb.set_tuning(bfs_words=0)


def test_determinism_repeat(P, sb):
    n, u, v, s = synth.rmat_two_faction(scale=12, m_target=1 << 15, seed=3)
    sb.load_graph(n, u, v, s)
    outs = []
    for _ in range(2):
        sb.sample_trees(4, 0, 1000)
        c, h = sb.frustration()
        outs.append((c.cpu().numpy(), h.cpu().numpy(), sb.label().cpu().numpy()))
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


# ------------------------------------------------------------------- cloud

def test_cloud_balanced_graph_single_state(P, sb):
    n, u, v, s, side = synth.planted_balanced(500, 900, seed=8)
    g = load_both(sb, n, u, v, s)
    sb.sample_trees(1, 0, 300)
    counts, _ = sb.frustration()
    assert int(counts.max()) == 0
    cl, fr = sb.cloud()
    assert cl["S"].tolist() == [0] and cl["count"].tolist() == [300] and fr == 0
    bits = sb.cloud_state(0).cpu().numpy().view(np.uint64)
    lab = ((bits[np.arange(g.n) // 64] >> (np.arange(g.n) % 64).astype(np.uint64)) & np.uint64(1)).astype(np.int8)
    assert np.array_equal(lab, (side ^ side[0]).astype(np.int8))


@pytest.mark.parametrize("fmax", [1, 5, 17, 400])
def test_scalable_cloud_matches_oracle(P, sb, fmax):
    """The scalable cloud over three sampling calls (130 + 130 + 140 trees)
    equals the oracle's on all 400 trees: same states, counts, S, first trees
    and hashes, in the same order; its states export like any other."""
    n, u, v, s = synth.random_connected(120, 260, neg_frac=0.35, seed=17)
    g = load_both(sb, n, u, v, s)
    sb.cloud_reset_scalable(fmax)
    t0 = 0
    for K in (130, 130, 140):
        sb.sample_trees(5, t0, K)
        sb.cloud_insert()
        t0 += K
    cl, fr = sb.cloud()
    ref = O.sample(g, 5, 0, t0)
    rc = O.cloud_bounded(ref["labels"], ref["counts"], fmax)
    assert np.array_equal(cl["first_tree"], rc["first_tree"])
    assert np.array_equal(cl["count"], rc["count"])
    assert np.array_equal(cl["S"], rc["S"])
    assert np.array_equal(cl["hash"], rc["H"])
    assert fr == int(rc["S"].min())
    for i in range(len(cl["S"])):
        st = sb.cloud_state(i).cpu().numpy().view(np.uint64)
        lab = ((st[np.arange(g.n) // 64] >> (np.arange(g.n) % 64).astype(np.uint64)) & np.uint64(1)).astype(np.uint8)
        assert np.array_equal(lab, ref["labels"][int(cl["first_tree"][i])])


def test_cloud_switch_lists_match_oracle(P, sb):
    """The edges each cloud state switches (the paper's output) equal the
    oracle's lab[u] ^ lab[v] ^ neg for that state's first tree, and their
    number is the state's S; the balanced state itself is sb_cloud_state."""
    n, u, v, s = synth.random_connected(400, 1300, neg_frac=0.3, seed=21)
    g = load_both(sb, n, u, v, s)
    seed, K = 3, 130
    sb.cloud_reset(max_states=K + 8)
    sb.sample_trees(seed, 0, K)
    cl, fr = sb.cloud()
    assert len(cl["S"]) > 10
    for i in range(len(cl["S"])):
        bits, cnt = sb.cloud_switch(i)
        _, _, clab, _ = O.tree(g, seed, int(cl["first_tree"][i]))
        want = (clab[g.eu] ^ clab[g.ev] ^ (g.eneg != 0)).astype(np.uint8)
        words = bits.cpu().numpy().view(np.uint64)
        got = ((words[np.arange(g.m) // 64] >> (np.arange(g.m) % 64).astype(np.uint64)) & np.uint64(1)).astype(np.uint8)
        assert np.array_equal(got, want), i
        assert cnt == int(want.sum()) == int(cl["S"][i])
        st = sb.cloud_state(i).cpu().numpy().view(np.uint64)
        lab = ((st[np.arange(g.n) // 64] >> (np.arange(g.n) % 64).astype(np.uint64)) & np.uint64(1)).astype(np.uint8)
        assert np.array_equal(lab, clab)
    assert fr == int(cl["S"].min())


@pytest.mark.parametrize("hash_bits", [64, 3])
def test_cloud_accumulates_and_checks_collisions(P, sb, hash_bits):
    # a small graph with few distinct states so trees repeat states
    n, u, v, s = synth.random_connected(12, 5, seed=21)
    g = load_both(sb, n, u, v, s)
    sb.cloud_reset(0, hash_bits)
    K = 150
    for t0 in (0, K, 2 * K):
        sb.sample_trees(2, t0, K)
        sb.cloud()
    cl, fr = sb.cloud()
    ref = O.sample(g, 2, 0, 3 * K)
    rc = O.cloud(ref["labels"], ref["counts"])
    assert np.array_equal(cl["first_tree"], rc["first_tree"])
    assert np.array_equal(cl["count"], rc["count"])
    assert np.array_equal(cl["S"], rc["S"])
    assert np.array_equal(cl["hash"], rc["H"])
    for i, f in enumerate(rc["first_tree"]):
        bits = sb.cloud_state(i).cpu().numpy().view(np.uint64)
        lab = ((bits[np.arange(g.n) // 64] >> (np.arange(g.n) % 64).astype(np.uint64)) & np.uint64(1)).astype(np.uint8)
        assert np.array_equal(lab, ref["labels"][f])


def test_cloud_capacity_error(P, sb):
    n, u, v, s = synth.random_connected(40, 60, seed=4)
    load_both(sb, n, u, v, s)
    sb.cloud_reset(2, 0)
    sb.sample_trees(0, 0, 64)
    with pytest.raises(P.SignedBalError) as e:
        sb.cloud(cap=2)
    assert e.value.code == -11


# ------------------------------------------------------------------ graphL

def _hub_graph(seed=31, n=900, extra=None, neg=0.3):
    """Vertex 0 joined to every other vertex, plus random distinct pairs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    extra = 2 * n if extra is None else extra
    a = np.concatenate([np.zeros(n - 1, np.int64), rng.integers(1, n, extra)])
    b = np.concatenate([np.arange(1, n), rng.integers(1, n, extra)])
    a, b = synth._unique_pairs_in_order(a, b)
    s = np.where(rng.random(a.shape[0]) < neg, -1, 1).astype(np.int8)
    return n, a, b, s


@pytest.mark.parametrize("R", [3, 8, 256])
def test_graphl_fwd_bwd_against_fp64(P, sb, R):
    n, a, b, s = _hub_graph()
    g = load_both(sb, n, a, b, s)
    gam = synth.gamma0(g.n, R, seed=R)
    G = torch.from_numpy(gam).cuda()
    loss, F = sb.graphL_fwd(G)
    L64, F64 = O.graphl_loss_f64(g, gam.astype(np.float64))
    assert np.array_equal(F.cpu().numpy(), F64)
    prod = np.abs(gam[g.eu].astype(np.float64) * gam[g.ev])
    bound = 1e-5 * (0.5 * (1.0 + prod)).sum(axis=0)
    assert np.all(np.abs(loss.cpu().numpy().astype(np.float64) - L64) <= bound)
    gout = torch.linspace(0.5, 1.5, R, device="cuda")
    grad = sb.graphL_bwd(G, gout).cpu().numpy().astype(np.float64)
    ref = O.graphl_grad_f64(g, gam.astype(np.float64), gout.cpu().numpy().astype(np.float64))
    assert np.linalg.norm(grad - ref) <= 1e-5 * np.linalg.norm(ref)
    absnb = np.zeros((g.n, R))
    np.add.at(absnb, g.eu, np.abs(gam[g.ev]))
    np.add.at(absnb, g.ev, np.abs(gam[g.eu]))
    comp_bound = 1e-5 * 0.5 * absnb * np.abs(gout.cpu().numpy())[None, :] + 1e-30
    assert np.all(np.abs(grad - ref) <= comp_bound)
    # bitwise reproducible
    assert torch.equal(sb.graphL_bwd(G, gout), sb.graphL_bwd(G, gout))


def test_graphl_segment_widths_give_identical_gradients(P, sb):
    """The graphL row kernel sums every row in the same fixed order whatever
    the width of its column segments (32, 64 or 128 columns), so the
    adjoint (Eq. 4) is bitwise the same for every lane knob, and within the
    float32 bound of the float64 oracle."""
    n, u, v, s = synth.rmat_two_faction(scale=11, m_target=1 << 14, seed=4)
    g = load_both(sb, n, u, v, s)
    R = 96
    gam = torch.from_numpy(synth.gamma0(g.n, R, seed=6)).cuda()
    gout = torch.from_numpy(np.random.default_rng(2).uniform(0.5, 2.0, R).astype(np.float32)).cuda()
    grads = {}
    for lanes in (8, 16, 32):
        sb.set_tuning(gl_lanes=lanes)
        grads[lanes] = sb.graphL_bwd(gam, gout).cpu().numpy()
    sb.set_tuning(gl_lanes=0)
    assert np.array_equal(grads[8], grads[16]) and np.array_equal(grads[8], grads[32])
    want = O.graphl_grad_f64(g, gam.cpu().numpy().astype(np.float64), gout.cpu().numpy().astype(np.float64))
    assert np.linalg.norm(grads[8] - want) <= 1e-5 * np.linalg.norm(want)


def test_graphl_autograd_function(P, sb):
    n, a, b, s = _hub_graph(seed=5, n=300)
    g = load_both(sb, n, a, b, s)
    gam = synth.gamma0(g.n, 4, seed=1)
    G = torch.from_numpy(gam).cuda().requires_grad_(True)
    loss = P.GraphLLoss.apply(G, sb)
    (loss * torch.tensor([1.0, 2.0, 3.0, 4.0], device="cuda")).sum().backward()
    ref = O.graphl_grad_f64(g, gam.astype(np.float64), np.array([1.0, 2.0, 3.0, 4.0]))
    got = G.grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


def test_graphl_descent_and_round(P, sb):
    n, a, b, s = _hub_graph(seed=9, n=600)
    g = load_both(sb, n, a, b, s)
    R, steps, alpha = 8, 90, 0.05
    gam = synth.gamma0(g.n, R, seed=2)
    G0 = torch.from_numpy(gam).cuda()
    out, exps, F_trace, F_final = sb.graphL_descent(G0, alpha, steps, renorm_log2=32, trace=True)
    ref, rexps, rtrace = O.graphl_descent_f64(g, gam, alpha, steps, renorm_log2=32, trace=True)
    e = exps.cpu().numpy()
    assert np.all(e > 0)  # the hub makes the update grow past 2^32
    got = out.cpu().numpy().astype(np.float64) * np.exp2(e.astype(np.float64))[None, :]
    want = ref * np.exp2(rexps.astype(np.float64))[None, :]
    scale = np.abs(want).max(axis=0)
    assert np.all(np.abs(got - want) <= 1e-3 * scale[None, :])
    # the first trace entry is the discrete loss of the start point, exactly
    assert np.array_equal(F_trace.cpu().numpy()[0], rtrace[0])
    # rounding: GPU and oracle agree exactly on the same float32 state
    Fr, flip = sb.graphL_round(out, want_flip=True)
    oF, oflip = O.graphl_round_f32(g, out.cpu().numpy(), want_flip=True)
    assert np.array_equal(Fr.cpu().numpy(), oF)
    assert np.array_equal(F_final.cpu().numpy(), oF)
    fw = flip.cpu().numpy().view(np.uint64)
    bits = ((fw[:, np.arange(g.m) // 64] >> (np.arange(g.m) % 64).astype(np.uint64)) & np.uint64(1)).astype(np.uint8)
    assert np.array_equal(bits, oflip)
    # final signs agree with the float64 run except where the value is tiny
    dis = np.sign(got) != np.sign(want)
    assert np.all(np.abs(want[dis]) <= 1e-3 * scale[np.nonzero(dis)[1]])


# ------------------------------------------------- full size, sampled trees

@pytest.fixture(scope="module")
def rmat20():
    """The 2^20-vertex, 2^24-edge two-faction R-MAT graph of the benchmark,
    raw and as the oracle cleans it."""
    n, u, v, s = synth.rmat_two_faction(scale=20, m_target=1 << 24)
    return (n, u, v, s), O.clean_graph(n, u, v, s)


def _oracle_trees(g, seed, trees, labels=True):
    """The oracle's trees `trees` of graph g, one tree per task on every host
    core: (counts, hashes, labels (len(trees), n) uint8 or None)."""
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        refs = list(ex.map(lambda t: O.sample(g, seed, int(t), 1, want_labels=labels), trees))
    counts = np.array([r["counts"][0] for r in refs], np.int32)
    hashes = np.array([r["hashes"][0] for r in refs], np.uint64)
    lab = np.stack([r["labels"][0] for r in refs]) if labels else None
    return counts, hashes, lab


def _label_bits(words, trees):
    """(n, W) label words -> (len(trees), n) uint8, bit t % 64 of word t // 64."""
    w = words.cpu().numpy().view(np.uint64)
    bits = np.unpackbits(w.view(np.uint8).reshape(w.shape[0], -1), axis=1, bitorder="little")
    return np.ascontiguousarray(bits[:, np.asarray(trees)].T)


def test_rmat_2pow20_sampled_trees(P, sb, rmat20):
    """The 2^20-vertex, 2^24-edge two-faction R-MAT graph in the benchmark's
    launch configuration (K = 1024 trees in one batch): every tree's count,
    state hash and labels, and the whole cloud, against the oracle bit for
    bit (Algorithm 1, Eq. 1)."""
    (n, u, v, s), g = rmat20
    n1, m1, _ = sb.load_graph(n, u, v, s)
    assert (n1, m1) == (g.n, g.m)
    K = 1024
    sb.cloud_reset(max_states=K + 64)
    sb.sample_trees(0, 0, K)
    counts, hashes = sb.frustration()
    counts, hashes = counts.cpu().numpy(), hashes.cpu().numpy().view(np.uint64)
    lab = _label_bits(sb.label(), range(K))
    cl, fr_min = sb.cloud()
    rc, rh, rlab = _oracle_trees(g, 0, range(K))
    assert np.array_equal(counts, rc)
    assert np.array_equal(hashes, rh)
    assert np.array_equal(lab, rlab)
    ref = O.cloud(rlab, rc)
    assert np.array_equal(cl["first_tree"], ref["first_tree"])
    assert np.array_equal(cl["count"], ref["count"])
    assert np.array_equal(cl["S"], ref["S"])
    assert np.array_equal(cl["hash"], ref["H"])
    assert fr_min == int(rc.min())


def test_rmat_2pow20_kruskal_sampled_trees(P, sb, rmat20):
    """Randomized Kruskal trees on the 2^20-vertex graph, 1024 in one call
    (two passes of trees): trees 5 and 1000, one per pass, against the oracle
    bit for bit."""
    (n, u, v, s), g = rmat20
    sb.load_graph(n, u, v, s)
    K = 1024
    sb.sample_trees_kruskal(2, 0, K)
    counts, hashes = sb.frustration()
    counts, hashes = counts.cpu().numpy(), hashes.cpu().numpy().view(np.uint64)
    labw = sb.label().cpu().numpy().view(np.uint64)
    for t in (5, 1000):
        k, _, clab = O.mst_tree(g, 2, t)
        assert k == g.n - 1
        assert counts[t] == O.frustration(g, clab)
        assert hashes[t] == np.uint64(O.state_hash(clab))
        lab = ((labw[:, t // 64] >> np.uint64(t % 64)) & np.uint64(1)).astype(np.uint8)
        assert np.array_equal(lab, clab)
    assert np.all(counts >= 0) and np.all(counts <= g.m - g.n + 1)


def test_graphl_gradient_central_differences_2000_vertex_subgraph(P, sb, rmat20):
    """The adjoint on a 2,000-vertex piece of the benchmark graph (the first
    2,000 vertices a BFS from vertex 0 reaches, their induced subgraph, its
    largest component) against float64 central differences of the oracle's
    relaxed loss (Eq. 3).  The loss is linear in every single coordinate, so
    the central difference is exact up to rounding; the float32 gradient
    must agree within 1e-5 relative (Eq. 4)."""
    import collections

    _, g = rmat20
    seen = np.full(g.n, -1, np.int64)
    seen[0] = 0
    order, dq = [0], collections.deque([0])
    while dq and len(order) < 2000:
        x = dq.popleft()
        for y in g.col[g.rowptr[x]:g.rowptr[x + 1]]:
            if seen[y] < 0 and len(order) < 2000:
                seen[y] = len(order)
                order.append(int(y))
                dq.append(int(y))
    keep = (seen[g.eu] >= 0) & (seen[g.ev] >= 0)
    su, sv = seen[g.eu[keep]].astype(np.int32), seen[g.ev[keep]].astype(np.int32)
    ss = np.where(g.eneg[keep] != 0, -1, 1).astype(np.int8)
    gs = load_both(sb, len(order), su, sv, ss)
    R = 8
    gam = synth.gamma0(gs.n, R, seed=3)
    gout = np.random.default_rng(9).uniform(0.5, 2.0, R).astype(np.float32)
    grad = sb.graphL_bwd(torch.from_numpy(gam).cuda(), torch.from_numpy(gout).cuda()).cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(13)
    vs, rs = rng.integers(0, gs.n, 64), rng.integers(0, R, 64)
    g64 = gam.astype(np.float64)
    fd = np.zeros(64)
    for i, (vv, rr) in enumerate(zip(vs, rs)):
        h = 1e-4 * max(1.0, abs(g64[vv, rr]))
        gp, gm = g64.copy(), g64.copy()
        gp[vv, rr] += h
        gm[vv, rr] -= h
        Lp, _ = O.graphl_loss_f64(gs, gp)
        Lm, _ = O.graphl_loss_f64(gs, gm)
        fd[i] = gout[rr] * (Lp[rr] - Lm[rr]) / (2 * h)
    got = grad[vs, rs]
    assert np.linalg.norm(got - fd) <= 1e-5 * np.linalg.norm(fd) + 1e-7


def test_graphl_config4_gradient_at_sampled_steps(P, sb, rmat20):
    """graphL on the 2^20-vertex benchmark graph with R = 256 start points
    and 500 descent steps at alpha = 0.05 (Alg. 2): at steps 0, 250 and 500
    the adjoint of the GPU's own Gamma (Eq. 4) is checked against the
    oracle's float64 gradient of that Gamma on 8 of the columns, within
    1e-5 relative in norm per column and the per-component bound of R12;
    the final discrete loss equals the oracle's exact count on the GPU's
    rounded states for every column."""
    (n, u, v, s), g = rmat20
    sb.load_graph(n, u, v, s)
    R, alpha = 256, 0.05
    g0 = torch.from_numpy(synth.gamma0(g.n, R, seed=0)).cuda()
    cols = np.array([0, 31, 64, 100, 128, 177, 200, 255])
    ones = torch.ones(R, device="cuda")
    for steps in (0, 250, 500):
        if steps:
            gam, exps, _, F_final = sb.graphL_descent(g0, alpha, steps)
        else:
            gam = g0
        grad = sb.graphL_bwd(gam, ones).cpu().numpy()[:, cols].astype(np.float64)
        gsub = np.ascontiguousarray(gam.cpu().numpy()[:, cols]).astype(np.float64)
        want = O.graphl_grad_f64(g, gsub)
        for j in range(len(cols)):
            assert np.linalg.norm(grad[:, j] - want[:, j]) <= 1e-5 * np.linalg.norm(want[:, j]), (steps, cols[j])
        # per component: |dg_v| <= 1e-5 * 1/2 * sum_j |G_j|
        absum = O.graphl_grad_f64(O.Graph(g.n, g.eu, g.ev, np.zeros(g.m, np.int8)), np.abs(gsub))
        assert np.all(np.abs(grad - want) <= 1e-5 * np.abs(absum) + 1e-30), steps
    F_ref, _ = O.graphl_round_f32(g, gam.cpu().numpy())
    assert np.array_equal(F_final.cpu().numpy(), F_ref)


def test_bounded_barrier_wait_times_out_and_the_context_recovers(P, sb):
    """The BFS grid barrier is a bounded wait.  With the stall test knob the
    barriers of one sampling call wait for a block that does not exist, so
    every wait runs out (after 20 ms here): the call's results are refused
    with SB_ERR_TIMEOUT, the knob resets itself, and the next call on the
    same context is exact again."""
    TIMEOUT = -12
    n, u, v, s = synth.random_connected(300, 900, seed=41)
    g = load_both(sb, n, u, v, s)
    sb.set_tuning(wait_us=20000, stall_test=1)
    sb.sample_trees(3, 0, 128)
    with pytest.raises(P.SignedBalError) as e:
        sb.frustration()
    assert e.value.code == TIMEOUT
    with pytest.raises(P.SignedBalError) as e:
        sb.label()
    assert e.value.code == TIMEOUT
    assert sb.get_tuning()["stall_test"] == 0
    sb.set_tuning(wait_us=0)
    check_batch(P, sb, g, seed=3, t0=0, K=128)
    check_batch(P, sb, g, seed=4, t0=7, K=200, parents=True)


def test_argument_and_state_errors(P):
    """Calls out of order and sizes out of range come back as status codes
    (no fault, no crash), and the context stays usable afterwards."""
    ARG, STATE = -1, -10
    sb = P.SignedBal(0)
    try:
        for call in (lambda: sb.sample_trees(0, 0, 8), lambda: sb.graph_edges()):
            with pytest.raises(P.SignedBalError) as e:
                call()
            assert e.value.code == STATE
        n, u, v, s = synth.random_connected(200, 500, seed=5)
        g = load_both(sb, n, u, v, s)
        with pytest.raises(P.SignedBalError) as e:
            sb.frustration()
        assert e.value.code == STATE
        for K in (0, 4097):
            with pytest.raises(P.SignedBalError) as e:
                sb.sample_trees(0, 0, K)
            assert e.value.code == ARG
        with pytest.raises(P.SignedBalError) as e:
            sb.sample_trees(0, -1, 8)
        assert e.value.code == ARG
        for knob, val in (("bfs_words", 33), ("bfs_group", 3), ("gl_lanes", 12), ("mst_words", 65), ("score_blocks_sm", 99),
                          ("wait_us", 60000001), ("stall_test", 2)):
            with pytest.raises(P.SignedBalError) as e:
                sb.set_tuning(**{knob: val})
            assert e.value.code == ARG
        # the largest K in one call, still exact
        check_batch(P, sb, g, seed=2, t0=0, K=4096, parents=False)
        sb.cloud_reset(max_states=5000)
        cl, _ = sb.cloud()
        with pytest.raises(P.SignedBalError) as e:
            sb.cloud_state(len(cl["S"]))
        assert e.value.code == ARG
        with pytest.raises(P.SignedBalError) as e:
            sb.cloud_switch(-1)
        assert e.value.code == ARG
        gam = torch.zeros((g.n, 4), device="cuda")
        for R in (0, 65537):
            with pytest.raises(P.SignedBalError) as e:
                sb._check(sb.lib.sb_graphL_fwd(sb.h, P._ptr(gam), R, P._ptr(gam), None))
            assert e.value.code == ARG
        # still usable
        check_batch(P, sb, g, seed=3, t0=5, K=70, parents=True)
    finally:
        sb.close()
