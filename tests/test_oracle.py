"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here touches the CUDA library.  Each test pins the oracle to a fact
that does not come from the oracle itself: the paper's worked example
(Fig. 1), known counts of digraph classes, the orbit-stabilizer identity,
brute force over all vertex subsets, closed forms on hand-worked graphs,
textbook invariants (triangles via a sparse matrix product) and the G(n,p)
expectation of Eq. 4.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.sparse as sp

from conftest import read_golden
from oracle import oracle as O
from paper_2201_11655_b300 import synth


def col_of(k, canon_mask):
    canon, _ = O.classes(k)
    hit = np.nonzero(canon == canon_mask)[0]
    assert hit.size == 1, canon_mask
    return int(hit[0])


# ---------------------------------------------------------------- classes --

def test_fig1_index_and_minimum():
    g = read_golden("fig1_motif_index.txt")
    k = int(g["k"][0])
    rows = g["rows"]
    bits = "".join(rows[i][j] for i in range(k) for j in range(k) if i != j)
    assert bits == g["bitstring"][0]
    idx = int(bits, 2)
    assert idx == int(g["index"][0])
    assert O.canonical_index(k, idx) == int(g["index_min"][0])


def test_fig1_isomorphs():
    # The three labelled isomorphs of the Fig. 1 motif are 53, 30 and 43; all
    # map to 30 and no other index does.
    members = [i for i in range(64) if O.canonical_index(3, i) == 30]
    assert members == [30, 43, 53]


def test_class_counts_known():
    # Weakly connected digraphs up to isomorphism on 3 / 4 nodes: 13 / 199
    # (OEIS A003085); all digraphs: 16 / 218 (OEIS A000273); labelled weakly
    # connected digraphs: 54 / 3834 (OEIS A003027).
    for k, nconn, nall, nlab in ((3, 13, 16, 54), (4, 199, 218, 3834)):
        canon, niso = O.classes(k)
        assert len(canon) == nconn
        assert int(niso.sum()) == nlab
        canon_all, niso_all = O.classes(k, connected_only=False)
        assert len(canon_all) == nall
        assert int(niso_all.sum()) == 2 ** (k * (k - 1))
        assert np.all(np.diff(canon) > 0)


def _matrix(k, idx):
    m = np.zeros((k, k), np.int64)
    b = k * (k - 1) - 1
    for i in range(k):
        for j in range(k):
            if i != j:
                m[i, j] = (idx >> b) & 1
                b -= 1
    return m


def test_orbit_stabilizer():
    # N_Iso(m) * |Aut(m)| = k! for every class (orbit-stabilizer theorem);
    # |Aut| is counted here directly on the adjacency matrix.
    for k in (3, 4):
        canon, niso = O.classes(k)
        for c, ni in zip(canon, niso):
            m = _matrix(k, int(c))
            aut = sum(1 for p in itertools.permutations(range(k))
                      if np.array_equal(m[np.ix_(p, p)], m))
            assert ni * aut == math.factorial(k)


def test_canonical_is_minimum_of_own_orbit():
    # Every index is >= its canonical index, and applying a permutation never
    # changes the canonical index.
    rng = np.random.default_rng(0)
    for k in (3, 4):
        for idx in rng.integers(0, 2 ** (k * (k - 1)), 200):
            c = O.canonical_index(k, int(idx))
            assert c <= idx
            m = _matrix(k, int(idx))
            p = rng.permutation(k)
            pm = m[np.ix_(p, p)]
            bits = "".join(str(pm[i, j]) for i in range(k) for j in range(k) if i != j)
            assert O.canonical_index(k, int(bits, 2)) == c


# ------------------------------------------------------- enumeration pins --

@pytest.mark.parametrize("k", [3, 4])
def test_esu_equals_brute_force_random(k):
    rng = np.random.default_rng(1234 + k)
    for trial in range(60):
        n = int(rng.integers(k, 14 if k == 4 else 22))
        p = float(rng.uniform(0.05, 0.6))
        n, s, d = synth.gnp(n, p, int(rng.integers(0, 2**31)))
        a, ga = O.count(n, s, d, k, threads=2)
        b, gb = O.count_brute(n, s, d, k)
        assert ga == gb
        np.testing.assert_array_equal(a, b)


def test_esu_equals_brute_force_gnp100():
    # The small benchmark workload itself, k = 3 and k = 4, two independent
    # enumerations.
    n, s, d = synth.gnp(100, 0.08, 0)
    for k in (3, 4):
        a, ga = O.count(n, s, d, k)
        b, gb = O.count_brute(n, s, d, k)
        assert ga == gb
        np.testing.assert_array_equal(a, b)


def test_self_loops_and_duplicates_ignored():
    n, s, d = synth.gnp(30, 0.2, 5)
    a, _ = O.count(n, s, d, 4)
    s2 = np.concatenate([s, s[:40], np.arange(10)])
    d2 = np.concatenate([d, d[:40], np.arange(10)])
    b, _ = O.count(n, s2, d2, 4)
    np.testing.assert_array_equal(a, b)


def test_csr_example_k3_hand_worked():
    # The CSR example graph: arcs 0>1 0>2 0>3 2>0 3>1 3>2.  Its four 3-sets are
    # all connected.  By hand: {0,1,2} is a mutual pair plus an out-arc
    # (minimum index 7), {0,1,3} a transitive triangle (11), {0,2,3} a mutual
    # pair plus a 2-path closing it (27), {1,2,3} an out-star from 3 (3).
    g = read_golden("csr_example.txt")
    arcs = [tuple(int(x) for x in a.split(">")) for a in g["arcs"]]
    s = np.array([a for a, _ in arcs]); d = np.array([b for _, b in arcs])
    out, found = O.count(4, s, d, 3)
    assert found == 4
    want = np.zeros((4, 13), np.uint64)
    for members, mask in (((0, 1, 2), 7), ((0, 1, 3), 11), ((0, 2, 3), 27), ((1, 2, 3), 3)):
        for v in members:
            want[v, col_of(3, mask)] += 1
    np.testing.assert_array_equal(out, want)
    out4, found4 = O.count(4, s, d, 4)
    assert found4 == 1
    # The whole graph is one 4-set.  Its minimum index, by hand: the first
    # (most significant) row wants no out-arc -- only vertex 1 has none -> 000;
    # the second wants no arc to vertex 1 -- only vertex 2 -> its arcs to the
    # last two positions: 3 before 0 makes them 0, 1 -> 001; then vertex 3
    # (arcs to 1 and 2, not to 0) -> 110; vertex 0 (arcs to all) -> 111:
    # 000 001 110 111 = 119.
    assert (out4[:, col_of(4, 119)] == 1).all() and out4.sum() == 4


def _arcs(pairs):
    pairs = list(pairs)
    return np.array([p[0] for p in pairs], np.int32), np.array([p[1] for p in pairs], np.int32)


@pytest.mark.parametrize("n", [4, 5, 7])
def test_complete_digraph(n):
    s, d = _arcs((i, j) for i in range(n) for j in range(n) if i != j)
    out3, _ = O.count(n, s, d, 3)
    out4, _ = O.count(n, s, d, 4)
    assert (out3[:, col_of(3, 63)] == math.comb(n - 1, 2)).all() and out3.sum() == n * math.comb(n - 1, 2)
    assert (out4[:, col_of(4, 4095)] == math.comb(n - 1, 3)).all() and out4.sum() == n * math.comb(n - 1, 3)


def test_directed_cycles():
    for n in (3, 4, 5, 8):
        s, d = _arcs((i, (i + 1) % n) for i in range(n))
        out3, _ = O.count(n, s, d, 3)
        if n == 3:
            assert (out3[:, col_of(3, 25)] == 1).all() and out3.sum() == 3
        else:
            # every vertex starts, ends and is the middle of one directed 2-path
            assert (out3[:, col_of(3, 6)] == 3).all() and out3.sum() == 3 * n
        if n >= 4:
            out4, _ = O.count(n, s, d, 4)
            if n == 4:
                assert (out4[:, col_of(4, 674)] == 1).all() and out4.sum() == 4
            else:
                assert (out4[:, col_of(4, 84)] == 4).all() and out4.sum() == 4 * n


@pytest.mark.parametrize("L", [3, 4, 9])
def test_stars(L):
    out_s, out_d = _arcs((0, i) for i in range(1, L + 1))
    n = L + 1
    for (s, d), m3, m4 in (((out_s, out_d), 3, 7), ((out_d, out_s), 10, 292)):
        o3, _ = O.count(n, s, d, 3)
        o4, _ = O.count(n, s, d, 4)
        c3, c4 = col_of(3, m3), col_of(4, m4)
        assert o3[0, c3] == math.comb(L, 2) and (o3[1:, c3] == L - 1).all()
        assert o3.sum() == 3 * math.comb(L, 2)
        assert o4[0, c4] == math.comb(L, 3) and (o4[1:, c4] == math.comb(L - 1, 2)).all()
        assert o4.sum() == 4 * math.comb(L, 3)


def test_transitive_tournament():
    # "regular DAG" of the toy-graph validations: i -> j for all i < j.
    n = 6
    s, d = _arcs((i, j) for i in range(n) for j in range(i + 1, n))
    o3, _ = O.count(n, s, d, 3)
    o4, _ = O.count(n, s, d, 4)
    assert (o3[:, col_of(3, 11)] == math.comb(n - 1, 2)).all() and o3.sum() == 3 * math.comb(n, 3)
    # every 4-set is a transitive tournament; its minimum index, by hand: the
    # sink first (row 000), then the vertex beating only the sink (100), then
    # the one beating those two (110), the source last (111): 000 100 110 111
    # = 311
    assert (o4[:, col_of(4, 311)] == math.comb(n - 1, 3)).all() and o4.sum() == 4 * math.comb(n, 4)


# ------------------------------------------------------------ invariants --

def _undirected(n, s, d):
    A = sp.coo_matrix((np.ones(s.size), (s, d)), shape=(n, n)).tocsr()
    U = ((A + A.T) > 0).astype(np.int64)
    U.setdiag(0)
    U.eliminate_zeros()
    return U.tocsr()


def test_k3_totals_and_triangles():
    # Connected 3-sets through v: C(d_v, 2) + sum_{a in N(v)} (d_a - 1) - 2 tri(v);
    # the classes whose G_U is a triangle sum to tri(v) = (U^2 o U)_vv / 2.
    n, s, d = synth.chung_lu(400, 4.0, 2.3, 7, reciprocity=0.3)
    U = _undirected(n, s, d)
    deg = np.asarray(U.sum(axis=1)).ravel()
    tri = np.asarray((U @ U).multiply(U).sum(axis=1)).ravel() // 2
    nbr_sum = U @ (deg - 1)
    out, found = O.count(n, s, d, 3)
    tot = out.sum(axis=1).astype(np.int64)
    np.testing.assert_array_equal(tot, deg * (deg - 1) // 2 + nbr_sum - 2 * tri)
    canon, _ = O.classes(3)
    # triangle classes: all three unordered pairs carry at least one arc
    tri_cols = []
    for c, m in enumerate(canon):
        M = _matrix(3, int(m))
        if all(M[i, j] or M[j, i] for i, j in ((0, 1), (0, 2), (1, 2))):
            tri_cols.append(c)
    np.testing.assert_array_equal(out[:, tri_cols].sum(axis=1).astype(np.int64), tri)
    assert out.sum() == 3 * found


def test_sum_over_vertices_is_k_times_global():
    n, s, d = synth.gnp(60, 0.1, 11)
    for k in (3, 4):
        out, found = O.count(n, s, d, k)
        assert int(out.sum()) == k * found


def _transpose_map(k):
    canon, _ = O.classes(k)
    m = {}
    for c, mask in enumerate(canon):
        M = _matrix(k, int(mask)).T
        bits = "".join(str(M[i, j]) for i in range(k) for j in range(k) if i != j)
        m[c] = col_of(k, O.canonical_index(k, int(bits, 2)))
    return np.array([m[c] for c in range(len(canon))])


def test_transpose_permutes_columns():
    n, s, d = synth.chung_lu(200, 3.0, 2.5, 3, reciprocity=0.2)
    for k in (3, 4):
        a, _ = O.count(n, s, d, k)
        b, _ = O.count(n, d, s, k)
        t = _transpose_map(k)
        want = np.zeros_like(a)
        want[:, t] = a
        np.testing.assert_array_equal(b, want)


def test_relabel_permutes_rows():
    n, s, d = synth.gnp(80, 0.07, 21)
    perm = np.random.default_rng(3).permutation(n).astype(np.int32)
    for k in (3, 4):
        a, _ = O.count(n, s, d, k)
        b, _ = O.count(n, perm[s], perm[d], k)
        np.testing.assert_array_equal(b[perm], a)


def test_disjoint_union_concatenates_rows():
    n1, s1, d1 = synth.gnp(40, 0.1, 1)
    n2, s2, d2 = synth.chung_lu(50, 3.0, 2.5, 2)
    a1, _ = O.count(n1, s1, d1, 4)
    a2, _ = O.count(n2, s2, d2, 4)
    b, _ = O.count(n1 + n2, np.concatenate([s1, s2 + n1]), np.concatenate([d1, d2 + n1]), 4)
    np.testing.assert_array_equal(b, np.vstack([a1, a2]))


def test_degree_rank_definition():
    n, s, d = synth.chung_lu(300, 3.0, 2.3, 9, reciprocity=0.2)
    U = _undirected(n, s, d)
    deg = np.asarray(U.sum(axis=1)).ravel()
    order = np.lexsort((np.arange(n), -deg))
    rank = O.degree_rank(n, s, d)
    np.testing.assert_array_equal(rank[order], np.arange(n))


def test_root_ranges_partition_the_count():
    # Lemma 1: a set is counted only from its lowest-ranked member, so disjoint
    # rank ranges partition the sets.
    n, s, d = synth.chung_lu(300, 3.0, 2.3, 13, reciprocity=0.2)
    rank = O.degree_rank(n, s, d)
    for k in (3, 4):
        full, gf = O.count(n, s, d, k)
        acc = np.zeros_like(full)
        tot = 0
        for lo, hi in ((0, 5), (5, 40), (40, 41), (41, n)):
            part, g = O.count_roots(n, s, d, k, rank, lo, hi)
            acc += part
            tot += g
        assert tot == gf
        np.testing.assert_array_equal(acc, full)
        # several ranges in one call == the sum of the single-range calls
        ranges = ((0, 5), (40, 41), (100, 160))
        multi, gm = O.count_root_ranges(n, s, d, k, rank, ranges)
        acc = np.zeros_like(full)
        tot = 0
        for lo, hi in ranges:
            part, g = O.count_roots(n, s, d, k, rank, lo, hi)
            acc += part
            tot += g
        assert gm == tot
        np.testing.assert_array_equal(multi, acc)


# ------------------------------------------------------- G(n,p), Eq. 4 --

@pytest.mark.parametrize("k,seeds", [(3, 200), (4, 60)])
def test_gnp_expectation_eq4(k, seeds):
    # Mean per-vertex local count over vertices and seeds of G(100, 0.08)
    # against Eq. 4 (exact by linearity of expectation).  Classes with a large
    # expectation: within 5 standard errors of the seed-to-seed spread.
    # Rare classes: the total over all seeds and vertices stays inside a
    # generous Poisson tail of the expected total.
    n, p = 100, 0.08
    E = O.gnp_expected_local(n, p, k)
    per_seed = []
    for seed in range(seeds):
        nn, s, d = synth.gnp(n, p, 10_000 + seed)
        out, _ = O.count(nn, s, d, k)
        per_seed.append(out.astype(np.float64).mean(axis=0))
    per_seed = np.array(per_seed)
    mean = per_seed.mean(axis=0)
    sd = per_seed.std(axis=0, ddof=1)
    big = E * n * seeds >= 200
    assert big.sum() >= 5
    se = sd[big] / math.sqrt(seeds)
    assert np.all(np.abs(mean[big] - E[big]) <= 5 * se + 1e-12), (mean[big], E[big], se)
    tot_obs = per_seed[:, ~big].sum(axis=0) * n
    tot_exp = E[~big] * n * seeds
    # observed totals are sums of per-vertex credits; each set credits k
    # vertices, so counts of sets are tot/k.  Poisson bound on sets.
    sets_obs = tot_obs / k
    sets_exp = tot_exp / k
    assert np.all(sets_obs <= sets_exp + 8 * np.sqrt(sets_exp) + 12)


# ----------------------------------------- undirected and per-edge modes --
# The undirected motifs of Tables 1-2 / Fig. 5 and the per-edge counts of the
# Discussion, pinned by an independent brute force written here in Python
# (its own class list, its own connectivity test), closed forms, the
# undirected form of Eq. 4 and counting identities.

import itertools


def _py_index(k, adj):
    idx = 0
    for i in range(k):
        for j in range(k):
            if i != j:
                idx = (idx << 1) | int(adj[i][j])
    return idx


def _py_canon(k, adj):
    return min(_py_index(k, [[adj[p[i]][p[j]] for j in range(k)] for i in range(k)])
               for p in itertools.permutations(range(k)))


def _py_classes(k, undirected):
    out = set()
    nb = k * (k - 1)
    for idx in range(1 << nb):
        adj = [[0] * k for _ in range(k)]
        b = nb - 1
        for i in range(k):
            for j in range(k):
                if i != j:
                    adj[i][j] = (idx >> b) & 1
                    b -= 1
        if undirected and any(adj[i][j] != adj[j][i] for i in range(k) for j in range(k)):
            continue
        und = [[adj[i][j] or adj[j][i] for j in range(k)] for i in range(k)]
        seen, stack = {0}, [0]
        while stack:
            x = stack.pop()
            for y in range(k):
                if und[x][y] and y not in seen:
                    seen.add(y)
                    stack.append(y)
        if len(seen) == k:
            out.add(_py_canon(k, adj))
    return sorted(out)


def _py_brute(n, s, d, k, undirected, per_edge):
    arcs = set(zip(s.tolist(), d.tolist())) - {(x, x) for x in range(n)}
    und = {(a, b) for a, b in arcs} | {(b, a) for a, b in arcs}
    cls = _py_classes(k, undirected)
    col = {m: i for i, m in enumerate(cls)}
    edges = sorted({(min(a, b), max(a, b)) for a, b in arcs})
    erow = {e: i for i, e in enumerate(edges)}
    out = np.zeros((len(edges) if per_edge else n, len(cls)), np.uint64)
    for S in itertools.combinations(range(n), k):
        seen, stack = {S[0]}, [S[0]]
        while stack:
            x = stack.pop()
            for y in S:
                if (x, y) in und and y not in seen:
                    seen.add(y)
                    stack.append(y)
        if len(seen) < k:
            continue
        rel = und if undirected else arcs
        adj = [[int(i != j and (S[i], S[j]) in rel) for j in range(k)] for i in range(k)]
        c = col[_py_canon(k, adj)]
        if per_edge:
            for i in range(k):
                for j in range(i + 1, k):
                    if (S[i], S[j]) in und:
                        out[erow[(S[i], S[j])], c] += 1
        else:
            for v in S:
                out[v, c] += 1
    return out


def test_undirected_class_counts():
    # connected graphs on 3 and 4 vertices: 2 and 6 (OEIS A001349); labelled
    # connected graphs: 4 and 38 (A001187)
    for k, nc, lab in ((3, 2, 4), (4, 6, 38)):
        canon, niso = O.classes_undirected(k)
        assert len(canon) == nc and int(niso.sum()) == lab
        assert canon.tolist() == _py_classes(k, True)
        # each undirected class is the directed class of its symmetric matrix
        assert set(canon.tolist()) <= set(O.classes(k)[0].tolist())
    assert O.classes(3)[0].tolist() == _py_classes(3, False)


@pytest.mark.parametrize("undirected,per_edge", [(True, False), (False, True), (True, True)])
def test_modes_match_python_brute_force(undirected, per_edge):
    rng = np.random.default_rng(7)
    for trial in range(14):
        n = int(rng.integers(4, 11))
        p = float(rng.uniform(0.15, 0.5))
        n, s, d = synth.gnp(n, p, 500 + trial)
        for k in (3, 4):
            want = _py_brute(n, s, d, k, undirected, per_edge)
            got, found = O.count_mode(n, s, d, k, undirected=undirected, per_edge=per_edge)
            np.testing.assert_array_equal(got, want, err_msg="trial %d k=%d" % (trial, k))


def _undirected_arcs(pairs):
    return (np.array([a for a, b in pairs], np.int32), np.array([b for a, b in pairs], np.int32))


def test_undirected_and_per_edge_closed_forms():
    cu3, cu4 = O.classes_undirected(3)[0].tolist(), O.classes_undirected(4)[0].tolist()
    tri, k4 = cu3.index(63), cu4.index(4095)
    path3 = cu3.index(23)
    # complete graph K_n (one arc per pair): every vertex in C(n-1,2) triangles / C(n-1,3) K4s
    for n in (5, 7):
        s, d = _undirected_arcs([(i, j) for i in range(n) for j in range(i + 1, n)])
        x3, _ = O.count_mode(n, s, d, 3, undirected=True)
        x4, _ = O.count_mode(n, s, d, 4, undirected=True)
        assert (x3[:, tri] == math.comb(n - 1, 2)).all() and x3.sum() == n * math.comb(n - 1, 2)
        assert (x4[:, k4] == math.comb(n - 1, 3)).all() and x4.sum() == n * math.comb(n - 1, 3)
        e3, _ = O.count_mode(n, s, d, 3, undirected=True, per_edge=True)
        e4, _ = O.count_mode(n, s, d, 4, undirected=True, per_edge=True)
        assert (e3[:, tri] == n - 2).all() and (e4[:, k4] == math.comb(n - 2, 2)).all()
    # star with L leaves: paths centre C(L,2), leaf L-1; 3-stars centre C(L,3), leaf C(L-1,2)
    L = 6
    s, d = _undirected_arcs([(0, i) for i in range(1, L + 1)])
    x3, _ = O.count_mode(L + 1, s, d, 3, undirected=True)
    assert x3[0, path3] == math.comb(L, 2) and (x3[1:, path3] == L - 1).all()
    x4, _ = O.count_mode(L + 1, s, d, 4, undirected=True)
    star = int(np.nonzero(x4[0])[0][0])
    assert x4[0, star] == math.comb(L, 3) and (x4[1:, star] == math.comb(L - 1, 2)).all()
    assert O.classes_undirected(4)[1][star] == 4  # the 3-star has 4 labellings
    e3, _ = O.count_mode(L + 1, s, d, 3, undirected=True, per_edge=True)
    e4, _ = O.count_mode(L + 1, s, d, 4, undirected=True, per_edge=True)
    assert (e3[:, path3] == L - 1).all() and (e4[:, star] == math.comb(L - 1, 2)).all()
    # cycle C_n, n >= 5: 3 paths and 4 four-paths through each vertex; 2 and 3 per edge
    n = 9
    s, d = _undirected_arcs([(i, (i + 1) % n) for i in range(n)])
    x3, _ = O.count_mode(n, s, d, 3, undirected=True)
    x4, _ = O.count_mode(n, s, d, 4, undirected=True)
    p4 = int(np.nonzero(x4[0])[0][0])
    assert (x3[:, path3] == 3).all() and (x4[:, p4] == 4).all() and O.classes_undirected(4)[1][p4] == 12
    e3, _ = O.count_mode(n, s, d, 3, undirected=True, per_edge=True)
    e4, _ = O.count_mode(n, s, d, 4, undirected=True, per_edge=True)
    assert (e3[:, path3] == 2).all() and (e4[:, p4] == 3).all()


@pytest.mark.parametrize("undirected", [False, True])
def test_per_edge_totals_identity(undirected):
    # every set of class m is credited to each of its e_m edges:
    # sum over edges of Y_m = e_m * (sum over vertices of X_m) / k
    n, s, d = synth.chung_lu(300, 3.0, 2.3, 21, reciprocity=0.3)
    for k in (3, 4):
        canon = (O.classes_undirected(k) if undirected else O.classes(k))[0]
        x, fx = O.count_mode(n, s, d, k, undirected=undirected)
        y, fy = O.count_mode(n, s, d, k, undirected=undirected, per_edge=True)
        assert fx == fy
        nedges = []
        for m in canon:
            bits = [(int(m) >> (k * (k - 1) - 1 - p)) & 1 for p in range(k * (k - 1))]
            adj = np.zeros((k, k), int)
            p = 0
            for i in range(k):
                for j in range(k):
                    if i != j:
                        adj[i, j] = bits[p]
                        p += 1
            nedges.append(int(((adj + adj.T) > 0).sum()) // 2)
        np.testing.assert_array_equal(y.sum(axis=0).astype(object),
                                      np.array(nedges, dtype=object) * x.sum(axis=0).astype(object) // k)
        # undirected rows sum to the same number of connected sets as directed ones
        xd, _ = O.count(n, s, d, k)
        np.testing.assert_array_equal(x.sum(axis=1), xd.sum(axis=1))


@pytest.mark.parametrize("k,seeds", [(3, 200), (4, 60)])
def test_undirected_gnp_expectation_eq4(k, seeds):
    # Eq. 4 with n_max = C(k, 2) on undirected G(100, 0.08)
    n, p = 100, 0.08
    E = O.gnp_expected_local(n, p, k, undirected=True)
    per_seed = []
    for seed in range(seeds):
        nn, s, d = synth.gnp_undirected(n, p, 20_000 + seed)
        out, _ = O.count_mode(nn, s, d, k, undirected=True)
        per_seed.append(out.astype(np.float64).mean(axis=0))
    per_seed = np.array(per_seed)
    mean = per_seed.mean(axis=0)
    sd = per_seed.std(axis=0, ddof=1)
    big = E * n * seeds >= 200
    assert big.sum() >= 2
    se = sd[big] / math.sqrt(seeds)
    assert np.all(np.abs(mean[big] - E[big]) <= 5 * se + 1e-12), (mean[big], E[big], se)
    sets_obs = per_seed[:, ~big].sum(axis=0) * n / k
    sets_exp = E[~big] * n * seeds / k
    assert np.all(sets_obs <= sets_exp + 8 * np.sqrt(sets_exp) + 12)
