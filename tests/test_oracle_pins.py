"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the paper's
worked example (Sec. 2, Fig. 1), exhaustive search (frustration index by
definition, max-cut for all-negative graphs, Sec. 1), Harary's theorem
(Sec. 2), the fundamental-cycle rule of the graphB+ algorithm (appendix),
library routines (scipy BFS distances, components, CSR, minimum spanning
trees; numpy matrix powers)
and closed forms (graphL's quadratic loss, Eq. 3-4).
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import synth
from tests._bruteforce import exact_frustration, max_cut

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _fig1():
    edges, meta = [], {}
    for line in open(os.path.join(GOLDEN, "paper_fig1.txt")):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] == "edge":
            edges.append((int(line[1]), int(line[2])))
        else:
            meta[line[0]] = int(line[1])
    return meta, np.array(edges, np.int32)


# ------------------------------------------------------------ hash primitives

def test_splitmix64_published_first_output(oracle):
    # SplitMix64 from state 0: the first output is the finaliser applied to the
    # golden-ratio increment; its published value is 0xE220A8397B1DCDAF.
    assert oracle.mix64(0x9E3779B97F4A7C15) == 0xE220A8397B1DCDAF


def test_hash_primitives_are_bijective_on_samples(oracle):
    xs = np.random.Generator(np.random.PCG64(5)).integers(0, 2**63, 20000, dtype=np.uint64)
    assert len({oracle.mix64(int(x)) for x in xs}) == len(set(int(x) for x in xs))
    assert len({oracle.fmix32(i) for i in range(20000)}) == 20000
    assert oracle.fmix32(0) == 0


def _murmur3_x86_32(data: bytes, seed: int, fmix) -> int:
    """MurmurHash3_x86_32 (Appleby, SMHasher): 4-byte little-endian blocks
    mixed with c1 = 0xcc9e2d51, c2 = 0x1b873593 and rotations by 15 and 13,
    the tail bytes, the length, then the 32-bit finaliser `fmix` under test."""
    M = 0xFFFFFFFF
    rotl = lambda x, r: ((x << r) | (x >> (32 - r))) & M
    c1, c2 = 0xCC9E2D51, 0x1B873593
    h = seed & M
    nb = len(data) // 4
    for i in range(nb):
        k = int.from_bytes(data[4 * i:4 * i + 4], "little")
        k = rotl((k * c1) & M, 15)
        h ^= (k * c2) & M
        h = (rotl(h, 13) * 5 + 0xE6546B64) & M
    tail = data[4 * nb:]
    if tail:
        k = int.from_bytes(tail, "little")
        k = rotl((k * c1) & M, 15)
        h ^= (k * c2) & M
    h ^= len(data)
    return fmix(h)


@pytest.mark.parametrize("data,seed,want", [
    (b"", 0, 0x00000000),
    (b"", 1, 0x514E28B7),  # = fmix32(1)
    (b"", 0xFFFFFFFF, 0x81F16F39),  # = fmix32(0xFFFFFFFF)
    (b"\0\0\0\0", 0, 0x2362F9DE),
    (b"aaaa", 0x9747B28C, 0x5A97808A),
    (b"abc", 0, 0xB3DD93FA),
    (b"Hello, world!", 0x9747B28C, 0x24884CBA),
    (b"The quick brown fox jumps over the lazy dog", 0x9747B28C, 0x2FA826CD),
])
def test_fmix32_gives_published_murmur3_vectors(oracle, data, seed, want):
    # The MurmurHash3 finaliser is the last step of MurmurHash3_x86_32; the
    # empty key reduces the whole hash to fmix32(seed).  Published test
    # vectors of the full hash therefore pin every constant and shift of it.
    assert _murmur3_x86_32(data, seed, oracle.fmix32) == want


def test_state_hash_is_a_subset_sum(oracle):
    rng = np.random.Generator(np.random.PCG64(9))
    n = 300
    a = (rng.random(n) < 0.3).astype(np.uint8)
    b = ((rng.random(n) < 0.3) & (a == 0)).astype(np.uint8)
    ha, hb, hab = oracle.state_hash(a), oracle.state_hash(b), oracle.state_hash(a | b)
    assert (ha + hb) % (1 << 64) == hab
    assert oracle.state_hash(np.zeros(n, np.uint8)) == 0


# ------------------------------------------------------------------ ingest

def test_clean_graph_matches_scipy_components_and_csr(oracle):
    rng = np.random.Generator(np.random.PCG64(3))
    n = 60
    a = rng.integers(0, n, 70)
    b = rng.integers(0, n, 70)
    keep = a != b
    a, b = a[keep], b[keep]
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    key = np.unique(lo * n + hi)
    lo, hi = key // n, key % n
    sign = np.where(rng.random(lo.shape[0]) < 0.4, -1, 1).astype(np.int8)
    g = oracle.clean_graph(n, lo, hi, sign)
    A = sp.coo_matrix((np.ones(lo.shape[0]), (lo, hi)), shape=(n, n))
    ncomp, lab = csg.connected_components(A, directed=False)
    sizes = np.bincount(lab)
    best = max(range(ncomp), key=lambda c: (sizes[c], -np.min(np.nonzero(lab == c)[0])))
    members = np.nonzero(lab == best)[0]
    assert g.n == members.shape[0]
    assert np.array_equal(np.nonzero(g.vmap >= 0)[0], members)
    assert np.array_equal(g.vmap[members], np.arange(g.n))
    # CSR against scipy's symmetric adjacency (sorted rows)
    S = sp.coo_matrix((np.ones(g.m), (g.eu, g.ev)), shape=(g.n, g.n))
    S = (S + S.T).tocsr()
    S.sort_indices()
    assert np.array_equal(g.rowptr, S.indptr)
    assert np.array_equal(g.col, S.indices)
    assert np.all(g.eu < g.ev)
    keys = g.eu.astype(np.int64) * g.n + g.ev
    assert np.all(np.diff(keys) > 0)


def test_clean_graph_errors(oracle):
    O = oracle
    with pytest.raises(O.OracleError) as e:
        O.clean_graph(3, [0, 1], [1, 1], [1, 1])
    assert e.value.code == -4  # self-loop
    with pytest.raises(O.OracleError) as e:
        O.clean_graph(3, [0, 1], [1, 2], [1, 0])
    assert e.value.code == -5  # invalid sign
    with pytest.raises(O.OracleError) as e:
        O.clean_graph(3, [0, 1], [1, 3], [1, 1])
    assert e.value.code == -9  # out of range
    with pytest.raises(O.OracleError) as e:
        O.clean_graph(3, [0, 1, 1], [1, 2, 0], [1, 1, -1])
    assert e.value.code == -6  # same pair, both signs
    with pytest.raises(O.OracleError) as e:
        O.clean_graph(3, [0, 1, 1], [1, 2, 0], [1, 1, 1], flags=O.LOAD_LCC)
    assert e.value.code == -7  # duplicate without merge
    g = O.clean_graph(3, [0, 1, 1], [1, 2, 0], [1, 1, 1])
    assert g.m == 2
    with pytest.raises(O.OracleError) as e:
        O.clean_graph(4, [0, 2], [1, 3], [1, 1], flags=O.LOAD_MERGE_DUP)
    assert e.value.code == -8  # disconnected without LCC
    g = O.clean_graph(4, [0, 2], [1, 3], [1, 1])
    assert g.n == 2 and list(g.vmap) == [0, 1, -1, -1]  # tie -> smallest id


# ------------------------------------------------------------ trees, labels

def _tree_checks(O, g, seed, t):
    root, parent, clab, level = O.tree(g, seed, t)
    A = sp.coo_matrix((np.ones(g.m), (g.eu, g.ev)), shape=(g.n, g.n))
    dist = csg.shortest_path(A, directed=False, unweighted=True, indices=root)
    assert np.array_equal(level, dist.astype(np.int32)), "levels are BFS distances"
    assert root == O.tree_root(seed, t, g.n)
    nb = {}
    for j in range(g.n):
        nb[j] = {int(c): int(s) for c, s in zip(g.col[g.rowptr[j]:g.rowptr[j + 1]],
                                                 g.colneg[g.rowptr[j]:g.rowptr[j + 1]])}
    tree_edges = 0
    for v in range(g.n):
        if v == root:
            assert parent[v] == -1
            continue
        p = int(parent[v])
        assert p in nb[v] and level[p] == level[v] - 1
        cands = [u for u in nb[v] if level[u] == level[v] - 1]
        assert p == min(cands, key=lambda u: O.parent_key(seed, t, u, v))
        tree_edges += 1
        # every tree edge is satisfied by the state
        assert clab[v] ^ clab[p] ^ nb[v][p] == 0
    assert tree_edges == g.n - 1
    # labels = parity of negative edges on the root path, vertex 0 canonical
    par_lab = np.zeros(g.n, np.uint8)
    for v in range(g.n):
        x, s = v, 0
        while x != root:
            s ^= nb[x][int(parent[x])]
            x = int(parent[x])
        par_lab[v] = s
    assert np.array_equal(clab, par_lab ^ par_lab[0])
    assert clab[0] == 0
    # graphB+ (appendix): S = number of non-tree edges with a negative
    # fundamental cycle, computed by walking both endpoints up to their LCA
    tree_set = {(min(v, int(parent[v])), max(v, int(parent[v]))) for v in range(g.n) if v != root}
    neg_cycles = 0
    for a, b, s in zip(g.eu, g.ev, g.eneg):
        if (int(a), int(b)) in tree_set:
            continue
        x, y, prod = int(a), int(b), int(s)
        while x != y:
            if level[x] >= level[y]:
                prod ^= nb[x][int(parent[x])]
                x = int(parent[x])
            else:
                prod ^= nb[y][int(parent[y])]
                y = int(parent[y])
        neg_cycles += prod
    assert g.m - len(tree_set) == g.m - g.n + 1  # Corollary, Sec. 2
    S = O.frustration(g, clab)
    assert S == neg_cycles
    return S, clab


@pytest.mark.parametrize("case", range(6))
def test_trees_labels_counts_on_random_graphs(oracle, case):
    n, u, v, s = synth.random_connected(9 + 3 * case, 6 + 4 * case, seed=100 + case)
    g = oracle.clean_graph(n, u, v, s)
    fr, _ = exact_frustration(g.n, g.eu, g.ev, g.eneg)
    for t in range(12):
        S, _ = _tree_checks(oracle, g, seed=case, t=t)
        assert S >= fr


def test_paper_example_all_sign_patterns(oracle):
    meta, E = _fig1()
    n = meta["vertices"]
    balanced_patterns = 0
    for pat in range(32):
        sign = np.array([-1 if (pat >> i) & 1 else 1 for i in range(5)], np.int8)
        g = oracle.clean_graph(n, E[:, 0], E[:, 1], sign)
        fr, nbal = exact_frustration(g.n, g.eu, g.ev, g.eneg)
        assert fr <= meta["max_frustration"]
        res = oracle.sample(g, seed=0, t0=0, K=32)
        cl = oracle.cloud(res["labels"], res["counts"])
        assert np.all(res["counts"] >= fr)
        if fr == 0:
            balanced_patterns += 1
            assert nbal == 1  # the unique bipartition, up to the global flip
            assert np.all(res["counts"] == 0)
            assert cl["S"].shape[0] == 1 and cl["count"][0] == 32
        else:
            assert res["counts"].min() == fr
    assert balanced_patterns == meta["balanced_patterns"]


@pytest.mark.parametrize("case", range(5))
def test_harary_planted_balance(oracle, case):
    n, u, v, s, side = synth.planted_balanced(10 + 2 * case, 10 + 3 * case, seed=200 + case)
    g = oracle.clean_graph(n, u, v, s)
    res = oracle.sample(g, seed=case, t0=0, K=24)
    assert np.all(res["counts"] == 0)
    cl = oracle.cloud(res["labels"], res["counts"])
    assert cl["S"].shape[0] == 1
    want = (side ^ side[0]).astype(np.uint8)
    assert np.array_equal(res["labels"][0], want)


@pytest.mark.parametrize("case", range(4))
def test_all_negative_maxcut(oracle, case):
    n, u, v, _ = synth.random_connected(8 + 2 * case, 8 + 2 * case, seed=300 + case)
    neg = -np.ones(u.shape[0], np.int8)
    g = oracle.clean_graph(n, u, v, neg)
    fr, _ = exact_frustration(g.n, g.eu, g.ev, g.eneg)
    assert fr == g.m - max_cut(g.n, g.eu, g.ev)  # Sec. 1: max-cut equivalence
    res = oracle.sample(g, seed=1, t0=0, K=16)
    assert np.all(res["counts"] >= fr)


def test_all_negative_bipartite_gives_zero(oracle):
    # even cycle + chords between the two colour classes: bipartite
    n = 10
    u = list(range(n))
    v = [(i + 1) % n for i in range(n)]
    u += [0, 2, 1]
    v += [3, 7, 4]
    neg = -np.ones(len(u), np.int8)
    g = oracle.clean_graph(n, u, v, neg)
    assert g.m - max_cut(g.n, g.eu, g.ev) == 0
    res = oracle.sample(g, seed=3, t0=0, K=20)
    assert np.all(res["counts"] == 0)


def test_parent_choice_is_randomized(oracle):
    # 4-cycle: the vertex opposite the root always has two candidate parents;
    # over many trees each candidate should win about half the time
    g = oracle.clean_graph(4, [0, 1, 2, 3], [1, 2, 3, 0], [1, 1, 1, 1])
    wins, total = 0, 0
    roots = np.zeros(4, int)
    for t in range(2000):
        root, parent, _, _ = oracle.tree(g, 11, t)
        roots[root] += 1
        opp = (root + 2) % 4
        wins += int(parent[opp] == min((opp + 1) % 4, (opp + 3) % 4))
        total += 1
    assert abs(wins / total - 0.5) < 0.05
    assert np.all(np.abs(roots / 2000 - 0.25) < 0.05)


# ------------------------------------------------- randomized Kruskal trees

def _mst_checks(O, g, seed, t):
    """One Kruskal tree against scipy's minimum spanning tree under the same
    weight order, and its labels against the tree (parity, canonical form)."""
    k, in_tree, clab = O.mst_tree(g, seed, t)
    assert k == g.n - 1 and int(in_tree.sum()) == g.n - 1
    # the minimum spanning tree depends only on the order of the weights:
    # ranks 1..m are exact in float64 and distinct
    w = np.array([O.mst_weight(seed, t, int(a), int(b)) for a, b in zip(g.eu, g.ev)], dtype=np.uint64)
    assert np.unique(w).shape[0] == g.m
    rank = np.empty(g.m, np.float64)
    rank[np.argsort(w, kind="stable")] = np.arange(1, g.m + 1)
    A = sp.coo_matrix((rank, (g.eu, g.ev)), shape=(g.n, g.n)).tocsr()
    T = csg.minimum_spanning_tree(A).tocoo()
    want = {(min(a, b), max(a, b)) for a, b in zip(T.row.tolist(), T.col.tolist())}
    got = {(int(a), int(b)) for a, b, x in zip(g.eu, g.ev, in_tree) if x}
    assert got == want
    # every tree edge satisfied; vertex 0 on the +1 side; spanning
    for a, b, s, x in zip(g.eu, g.ev, g.eneg, in_tree):
        if x:
            assert clab[a] ^ clab[b] ^ s == 0
    assert clab[0] == 0
    Tm = sp.coo_matrix((np.ones(g.n - 1), ([a for a, _ in got], [b for _, b in got])), shape=(g.n, g.n))
    assert csg.connected_components(Tm, directed=False)[0] == 1
    return O.frustration(g, clab), clab


@pytest.mark.parametrize("case", range(4))
def test_kruskal_trees_are_minimum_spanning_trees(oracle, case):
    n, u, v, s = synth.random_connected(9 + 4 * case, 8 + 5 * case, seed=500 + case)
    g = oracle.clean_graph(n, u, v, s)
    fr, _ = exact_frustration(g.n, g.eu, g.ev, g.eneg)
    res = oracle.mst_sample(g, seed=case, t0=0, K=10, want_in_tree=True)
    for t in range(10):
        S, clab = _mst_checks(oracle, g, case, t)
        assert S >= fr
        assert res["counts"][t] == S and np.array_equal(res["labels"][t], clab)
        assert res["hashes"][t] == np.uint64(oracle.state_hash(clab))


def test_kruskal_tree_equals_prims_tree(oracle):
    """Prim's algorithm (the appendix's other weighted sampler) grown from
    vertex 0 on the same weights gives the same tree: with distinct weights
    the minimum spanning tree is unique."""
    import heapq

    n, u, v, s = synth.random_connected(30, 60, seed=808)
    g = oracle.clean_graph(n, u, v, s)
    adj = [[] for _ in range(g.n)]
    for e, (a, b) in enumerate(zip(g.eu.tolist(), g.ev.tolist())):
        adj[a].append((b, e))
        adj[b].append((a, e))
    for t in range(8):
        w = [oracle.mst_weight(3, t, a, b) for a, b in zip(g.eu.tolist(), g.ev.tolist())]
        inside, heap, tree = {0}, [(w[e], e, y) for y, e in adj[0]], set()
        heapq.heapify(heap)
        while heap:
            _, e, y = heapq.heappop(heap)
            if y in inside:
                continue
            inside.add(y)
            tree.add(e)
            for z, f in adj[y]:
                if z not in inside:
                    heapq.heappush(heap, (w[f], f, z))
        _, in_tree, _ = oracle.mst_tree(g, 3, t)
        assert set(np.nonzero(in_tree)[0].tolist()) == tree


def test_kruskal_tree_distribution_on_k4_matches_random_edge_orders(oracle):
    """On the complete graph K4 the hashed weights must act like a uniformly
    random edge order: the frequency of each of the 16 spanning trees over
    20,000 trees matches the exact law of Kruskal's algorithm over all 720
    edge orders (brute force), within 4 standard deviations."""
    import itertools

    eu = [0, 0, 0, 1, 1, 2]
    ev = [1, 2, 3, 2, 3, 3]
    g = oracle.clean_graph(4, eu, ev, [1] * 6)
    exact = {}
    for order in itertools.permutations(range(6)):
        comp, tree = list(range(4)), []
        for e in order:
            a, b = comp[g.eu[e]], comp[g.ev[e]]
            if a != b:
                comp = [a if c == b else c for c in comp]
                tree.append(e)
        key = tuple(sorted(tree))
        exact[key] = exact.get(key, 0) + 1
    assert len(exact) == 16 and sum(exact.values()) == 720
    K = 20000
    got = oracle.mst_sample(g, seed=21, t0=0, K=K, want_labels=False, want_in_tree=True)["in_tree"]
    seen = {}
    for row in got:
        key = tuple(np.nonzero(row)[0].tolist())
        seen[key] = seen.get(key, 0) + 1
    assert set(seen) == set(exact)
    for key, cnt in exact.items():
        p = cnt / 720
        assert abs(seen[key] - K * p) <= 4 * np.sqrt(K * p * (1 - p)), (key, seen[key], K * p)


def test_kruskal_harary_planted_balance(oracle):
    n, u, v, s, side = synth.planted_balanced(16, 20, seed=601)
    g = oracle.clean_graph(n, u, v, s)
    res = oracle.mst_sample(g, seed=4, t0=0, K=16)
    assert np.all(res["counts"] == 0)
    want = (side ^ side[0]).astype(np.uint8)
    assert all(np.array_equal(lab, want) for lab in res["labels"])


def test_kruskal_cycle_drops_each_edge_equally_often(oracle):
    # a 5-cycle: the tree omits the heaviest edge, which is uniform over the
    # five edges when the weights are random
    g = oracle.clean_graph(5, [0, 1, 2, 3, 4], [1, 2, 3, 4, 0], [1, -1, 1, 1, -1])
    res = oracle.mst_sample(g, seed=9, t0=0, K=5000, want_labels=False, want_in_tree=True)
    assert np.all(res["in_tree"].sum(axis=1) == 4)
    freq = 1.0 - res["in_tree"].mean(axis=0)
    assert np.all(np.abs(freq - 0.2) < 0.02)
    # two negative edges make the cycle positive: balanced, S = 0 for every
    # tree; with one negative edge the omitted edge closes a negative cycle
    assert np.all(res["counts"] == 0)
    g1 = oracle.clean_graph(5, [0, 1, 2, 3, 4], [1, 2, 3, 4, 0], [1, -1, 1, 1, 1])
    assert np.all(oracle.mst_sample(g1, seed=9, t0=0, K=200)["counts"] == 1)


# ------------------------------------------------------------------ cloud

def test_cloud_invariants_and_sharding(oracle):
    n, u, v, s = synth.random_connected(14, 10, seed=41)
    g = oracle.clean_graph(n, u, v, s)
    K = 64
    res = oracle.sample(g, seed=2, t0=0, K=K)
    cl = oracle.cloud(res["labels"], res["counts"])
    assert cl["count"].sum() == K
    assert np.all(np.diff(cl["first_tree"]) > 0)
    for f, S, H in zip(cl["first_tree"], cl["S"], cl["H"]):
        assert S == oracle.frustration(g, res["labels"][f])
        assert H == oracle.state_hash(res["labels"][f])
    # distinct states
    reps = res["labels"][cl["first_tree"]]
    assert len({r.tobytes() for r in reps}) == reps.shape[0]
    # sharding: the halves, merged by state, give the whole
    a = oracle.sample(g, seed=2, t0=0, K=K // 2)
    b = oracle.sample(g, seed=2, t0=K // 2, K=K // 2)
    assert np.array_equal(np.concatenate([a["labels"], b["labels"]]), res["labels"])
    ca = oracle.cloud(a["labels"], a["counts"], t0=0)
    cb = oracle.cloud(b["labels"], b["counts"], t0=K // 2)
    merged = {}
    for c, lab in ((ca, a["labels"]), (cb, b["labels"])):
        for i in range(c["S"].shape[0]):
            key = lab[c["first_tree"][i] - (0 if c is ca else K // 2)].tobytes()
            f, cnt = merged.get(key, (1 << 60, 0))
            merged[key] = (min(f, int(c["first_tree"][i])), cnt + int(c["count"][i]))
    whole = {res["labels"][f].tobytes(): (int(f), int(c)) for f, c in zip(cl["first_tree"], cl["count"])}
    assert merged == whole


# ------------------------------------------------------------------ graphL

def _small_graph(oracle, seed=5):
    n, u, v, s = synth.random_connected(12, 14, seed=seed)
    return oracle.clean_graph(n, u, v, s)


def _scalable_case(O, K=400, seed=17):
    n, u, v, s = synth.random_connected(120, 260, neg_frac=0.35, seed=seed)
    g = O.clean_graph(n, u, v, s)
    smp = O.sample(g, 5, 0, K)
    return smp, O.cloud(smp["labels"], smp["counts"])


def test_scalable_cloud_without_eviction_follows_the_first_state(oracle):
    """With room for every state, the scalable cloud (appendix algorithm
    alg-scale) holds the first tree's state, counted once (its repeats are
    not below the largest stored S), followed by every state whose S is below
    it with all its trees, in order of first appearance; nothing else.
    Derived from the unbounded cloud."""
    smp, full = _scalable_case(oracle)
    K = smp["counts"].shape[0]
    b = oracle.cloud_bounded(smp["labels"], smp["counts"], fmax=K)
    s0 = int(full["S"][0])
    keep = full["S"] < s0
    assert full["first_tree"][0] == 0
    assert b["first_tree"].tolist() == [0] + full["first_tree"][keep].tolist()
    assert b["count"].tolist() == [1] + full["count"][keep].tolist()
    assert b["S"].tolist() == [s0] + full["S"][keep].tolist()
    assert np.array_equal(b["H"], np.concatenate([full["H"][:1], full["H"][keep]]))
    assert keep.sum() >= 3  # the case exercises the rule


def test_scalable_cloud_single_slot_keeps_the_first_minimum(oracle):
    """fmax = 1: the one slot ends with the first tree whose S is the minimum
    over all trees, counted once."""
    smp, _ = _scalable_case(oracle, seed=18)
    b = oracle.cloud_bounded(smp["labels"], smp["counts"], fmax=1)
    c = smp["counts"]
    assert b["S"].tolist() == [int(c.min())]
    assert b["first_tree"].tolist() == [int(np.argmin(c))]
    assert b["count"].tolist() == [1]


@pytest.mark.parametrize("fmax", [2, 5, 17])
def test_scalable_cloud_with_eviction_invariants(oracle, fmax):
    """With eviction: at most fmax states, all of them states of the
    unbounded cloud with no more trees than there, and the minimum S over
    all trees always kept (the evicted state is one with the largest S)."""
    smp, full = _scalable_case(oracle, seed=19)
    b = oracle.cloud_bounded(smp["labels"], smp["counts"], fmax=fmax)
    assert 1 <= len(b["S"]) <= fmax
    assert int(b["S"].min()) == int(smp["counts"].min())
    by_h = {int(h): (int(c), int(s_)) for h, c, s_ in zip(full["H"], full["count"], full["S"])}
    for h, c, s_ in zip(b["H"], b["count"], b["S"]):
        assert int(h) in by_h
        assert c <= by_h[int(h)][0] and s_ == by_h[int(h)][1]
    assert len(b["S"]) == fmax  # the case fills the cloud, so eviction happened


def test_scalable_cloud_evicts_the_lowest_slot_of_largest_S(oracle):
    """A hand-built tree sequence for the scalable cloud (appendix algorithm
    alg-scale, R14 reading) with fmax = 3, where the largest stored S is held
    by two slots twice.  Walking the rule by hand (slot contents after each
    tree):
      t0 A9 -> [A9]          t1 B7 -> [A9 B7]        t2 C7 -> [A9 B7 C7]
      t3 D6 -> [D6 B7 C7]    (replaces the one largest, A9)
      t4 E5 -> [D6 E5 C7]    (B7 and C7 tie: the lower slot, B, goes)
      t5 F4 -> [D6 E5 F4]    t6 G4 -> [G4 E5 F4]     t7 H3 -> [G4 H3 F4]
      t8 I2 -> [I2 H3 F4]    (G4 and F4 tie: the lower slot, G, goes)
      t9 F4 -> not below the largest S (4): not counted
      t10 H3 -> below 4 and stored: H counted twice
    Output by storing tree: F (t5), H (t7), I (t8).  Evicting the higher slot
    among equals would end with G (t6), H (t7), I (t8) instead."""
    n = 6
    states = {}
    for name in "ABCDEFGHI":  # distinct canonical labellings (vertex 0 on the +1 side)
        i = "ABCDEFGHI".index(name) + 1
        states[name] = np.array([0] + [(i >> b) & 1 for b in range(n - 1)], np.uint8)
    seq = [("A", 9), ("B", 7), ("C", 7), ("D", 6), ("E", 5), ("F", 4), ("G", 4), ("H", 3), ("I", 2),
           ("F", 4), ("H", 3)]
    labels = np.stack([states[a] for a, _ in seq])
    counts = np.array([c for _, c in seq], np.int32)
    b = oracle.cloud_bounded(labels, counts, fmax=3, t0=100)
    assert b["first_tree"].tolist() == [105, 107, 108]
    assert b["S"].tolist() == [4, 3, 2]
    assert b["count"].tolist() == [1, 2, 1]
    assert [int(h) for h in b["H"]] == [oracle.state_hash(states[x]) for x in "FHI"]


def test_graphl_gradient_central_differences(oracle):
    g = _small_graph(oracle)
    R = 3
    gam = synth.gamma0(g.n, R, seed=1).astype(np.float64)
    grad = oracle.graphl_grad_f64(g, gam)
    h = 1e-3
    for v in range(g.n):
        for r in range(R):
            gp = gam.copy(); gp[v, r] += h
            gm = gam.copy(); gm[v, r] -= h
            Lp, _ = oracle.graphl_loss_f64(g, gp)
            Lm, _ = oracle.graphl_loss_f64(g, gm)
            fd = (Lp[r] - Lm[r]) / (2 * h)  # exact for a function linear in gam[v, r]
            assert abs(fd - grad[v, r]) <= 1e-9 * (1 + abs(grad[v, r]))


def test_graphl_loss_closed_forms(oracle):
    g = _small_graph(oracle, seed=6)
    rng = np.random.Generator(np.random.PCG64(2))
    theta = np.where(rng.random((g.n, 4)) < 0.5, -1.0, 1.0)
    L, F = oracle.graphl_loss_f64(g, theta)
    assert np.array_equal(L, F.astype(np.float64))  # Eq. 3 at theta in {+-1} is Eq. 2
    Fr, flip = oracle.graphl_round_f32(g, theta.astype(np.float32), want_flip=True)
    assert np.array_equal(Fr, F)
    assert np.array_equal(flip.sum(axis=1), F)
    fr, _ = exact_frustration(g.n, g.eu, g.ev, g.eneg)
    assert np.all(F >= fr)
    # zero state: every edge contributes 1/2
    L0, _ = oracle.graphl_loss_f64(g, np.zeros((g.n, 2)))
    assert np.all(L0 == g.m / 2)
    # the loss equals m/2 - 1/2 G^T A_sigma G / 2 with A_sigma the signed adjacency
    A = np.zeros((g.n, g.n))
    for a, b, s in zip(g.eu, g.ev, g.eneg):
        A[a, b] = A[b, a] = -1.0 if s else 1.0
    gam = synth.gamma0(g.n, 2, seed=4).astype(np.float64)
    L, _ = oracle.graphl_loss_f64(g, gam)
    want = g.m / 2 - 0.25 * np.einsum("ir,ij,jr->r", gam, A, gam)
    assert np.allclose(L, want, rtol=1e-12, atol=1e-12)


def test_graphl_descent_is_a_matrix_power(oracle):
    g = _small_graph(oracle, seed=7)
    A = np.zeros((g.n, g.n))
    for a, b, s in zip(g.eu, g.ev, g.eneg):
        A[a, b] = A[b, a] = -1.0 if s else 1.0
    alpha, steps = 0.05, 40
    gam0 = synth.gamma0(g.n, 3, seed=8).astype(np.float64)
    out, exps, _ = oracle.graphl_descent_f64(g, gam0, alpha, steps, renorm_log2=0)
    want = np.linalg.matrix_power(np.eye(g.n) + 0.5 * alpha * A, steps) @ gam0
    assert np.allclose(out, want, rtol=1e-10, atol=1e-12)
    assert np.all(exps == 0)


def _signed_adjacency(g):
    A = np.zeros((g.n, g.n))
    for a, b, s in zip(g.eu, g.ev, g.eneg):
        A[a, b] = A[b, a] = -1.0 if s else 1.0
    return A


U32 = 2.0**-24  # unit roundoff of float32


def test_graphl_grad_f32_within_its_rounding_bound(oracle):
    """Eq. 4 in float32: each component is a sequential sum of deg(v) terms
    times -1/2 and the upstream weight, so it lies within
    (deg(v) + 1) u * 1/2 |gout| sum_j |G_j| of the float64 gradient (standard
    bound of recursive summation, u = 2^-24).  The float64 gradient is pinned
    by central differences above; here it is also recomputed as
    -1/2 A_sigma G with numpy."""
    g = _small_graph(oracle, seed=11)
    R = 5
    gam = synth.gamma0(g.n, R, seed=12)
    gout = np.array([1.0, -2.0, 0.5, 3.0, 0.25], np.float32)
    A = _signed_adjacency(g)
    g64 = oracle.graphl_grad_f64(g, gam.astype(np.float64), gout.astype(np.float64))
    assert np.allclose(g64, -0.5 * (A @ gam.astype(np.float64)) * gout[None, :], rtol=1e-12, atol=1e-14)
    g32 = oracle.graphl_grad_f32(g, gam, gout)
    deg = np.abs(A).sum(axis=1)
    bound = (deg[:, None] + 1) * U32 * 0.5 * np.abs(gout)[None, :] * (np.abs(A) @ np.abs(gam.astype(np.float64)))
    assert np.all(np.abs(g32.astype(np.float64) - g64) <= bound * 1.0001 + 1e-30)
    # the norm-wise contract of the float32 path
    assert np.linalg.norm(g32 - g64) <= 1e-5 * np.linalg.norm(g64)
    # sign: with every edge positive and G > 0 the gradient is negative (Eq. 4)
    pos = oracle.Graph(g.n, g.eu, g.ev, np.zeros(g.m, np.int8))
    gp = oracle.graphl_grad_f32(pos, np.abs(gam) + 0.5)
    assert np.all(gp < 0)


def test_graphl_descent_f32_follows_the_matrix_power_within_its_bound(oracle):
    """Alg. 2 in float32: lambda updates G <- G - alpha dL/dG are lambda
    products with B = I + alpha/2 A_sigma.  Each float32 update adds an error
    of at most (deg + 3) u (|B| |G|) per component, so after lambda steps
    |G32 - B^lambda G0| <= lambda (dmax + 3) u |B|^lambda |G0| to first
    order (a 1 % margin covers the second-order terms)."""
    g = _small_graph(oracle, seed=13)
    A = _signed_adjacency(g)
    alpha, steps = 0.05, 40
    gam0 = synth.gamma0(g.n, 4, seed=14)
    out, exps = oracle.graphl_descent_f32(g, gam0, alpha, steps, renorm_log2=0)
    assert np.all(exps == 0)
    B = np.eye(g.n) + 0.5 * alpha * A
    want = np.linalg.matrix_power(B, steps) @ gam0.astype(np.float64)
    dmax = np.abs(A).sum(axis=1).max()
    bound = steps * (dmax + 3) * U32 * (np.linalg.matrix_power(np.abs(B), steps) @ np.abs(gam0.astype(np.float64)))
    err = np.abs(out.astype(np.float64) - want)
    assert np.all(err <= 1.01 * bound)
    # the bound is tight enough to catch a sign error in the update
    wrong = np.linalg.matrix_power(np.eye(g.n) - 0.5 * alpha * A, steps) @ gam0.astype(np.float64)
    assert np.any(np.abs(out.astype(np.float64) - wrong) > 1.01 * bound)
    # with renormalisation: signs and values up to the recorded power of two
    out2, exps2 = oracle.graphl_descent_f32(g, gam0, 0.9, 30, renorm_log2=4)
    ref2 = np.linalg.matrix_power(np.eye(g.n) + 0.45 * A, 30) @ gam0.astype(np.float64)
    assert np.all(exps2 > 0)
    scaled = out2.astype(np.float64) * np.exp2(exps2.astype(np.float64))[None, :]
    big = np.abs(ref2) > 1e-3 * np.abs(ref2).max(axis=0, keepdims=True)
    assert np.array_equal(np.sign(scaled[big]), np.sign(ref2[big]))
    assert np.allclose(scaled, ref2, rtol=1e-4, atol=1e-4 * np.abs(ref2).max())


def test_graphl_renorm_keeps_signs(oracle):
    g = _small_graph(oracle, seed=9)
    gam0 = synth.gamma0(g.n, 4, seed=10)
    a, ea, _ = oracle.graphl_descent_f64(g, gam0, 0.9, 60, renorm_log2=0)
    b, eb, _ = oracle.graphl_descent_f64(g, gam0, 0.9, 60, renorm_log2=8)
    assert np.all(eb > 0)
    assert np.array_equal(np.sign(a), np.sign(b))
    assert np.array_equal(a, b * np.exp2(eb.astype(np.float64))[None, :])  # exact powers of two
    c, ec = oracle.graphl_descent_f32(g, gam0, 0.9, 60, renorm_log2=8)
    d, ed = oracle.graphl_descent_f32(g, gam0, 0.9, 60, renorm_log2=16)
    assert np.array_equal(np.sign(c), np.sign(d))
