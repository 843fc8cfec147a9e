"""GPU parity of the undirected variant and of per-edge counts (Tables 1-2's
undirected motifs; the Discussion's edge counts) against the oracle's modes,
bit for bit, through every kernel route (warp-per-task, root-per-CTA, split
roots)."""
import numpy as np
import pytest

from gpu_util import to_numpy_u64
from oracle import oracle as O
from paper_2201_11655_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SCHEDULES = [dict(hub_min_l=0), dict(hub_min_l=1), dict(hub_min_l=4, hub_split=3, hub_split_roots=6, hub_warps=32),
             dict(hub_min_l=2, d3_bits=64)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_11655_b300 import build, vdmc
    build.build()
    vdmc.load()
    old = vdmc.get_schedule()
    yield
    vdmc.set_schedule(**old)


def graphs():
    yield synth.gnp(100, 0.08, 0)
    yield synth.gnp_undirected(60, 0.15, 3)
    for i in range(6):
        yield synth.gnp(int(20 + 13 * i), 0.05 + 0.03 * i, 900 + i)
    yield synth.chung_lu(1500, 3.0, 2.2, 31, reciprocity=0.3)


@pytest.mark.parametrize("sched", SCHEDULES)
def test_undirected_counts_vs_oracle(sched):
    from paper_2201_11655_b300 import vdmc
    vdmc.set_schedule(**sched)
    for n, s, d in graphs():
        with vdmc.graph_create(n, s, d, undirected=True) as g:
            for k in (3, 4):
                assert g.num_classes(k) == (2 if k == 3 else 6)
                got = to_numpy_u64(vdmc.count(g, k))
                torch.cuda.synchronize()
                assert g.device_status() == 0
                want, _ = O.count_mode(n, s, d, k, undirected=True)
                np.testing.assert_array_equal(got, want, err_msg="undirected k=%d n=%d %s" % (k, n, sched))


@pytest.mark.parametrize("undirected", [False, True])
def test_per_edge_counts_vs_oracle(undirected):
    from paper_2201_11655_b300 import vdmc
    for n, s, d in graphs():
        with vdmc.graph_create(n, s, d, undirected=undirected) as g:
            u, v, f = g.edges()
            ou, ov = O.edges(n, s, d)
            np.testing.assert_array_equal(u, ou)
            np.testing.assert_array_equal(v, ov)
            arcs = set(zip(s.tolist(), d.tolist()))
            for i in range(len(u)):
                # an undirected graph takes every edge as arcs both ways
                want_f = 3 if undirected else ((u[i], v[i]) in arcs) + 2 * ((v[i], u[i]) in arcs)
                assert int(f[i]) == want_f
            for k in (3, 4):
                got = to_numpy_u64(vdmc.count_edges(g, k))
                torch.cuda.synchronize()
                assert g.device_status() == 0
                want, _ = O.count_mode(n, s, d, k, undirected=undirected, per_edge=True)
                np.testing.assert_array_equal(got, want, err_msg="per-edge k=%d n=%d undirected=%s" % (
                    k, n, undirected))
            # vertex counts on the same graph are unchanged by an edge count
            # in between (shared cursor and status word)
            x = to_numpy_u64(vdmc.count(g, 3))
            want, _ = O.count_mode(n, s, d, 3, undirected=undirected)
            np.testing.assert_array_equal(x, want)


def test_per_edge_totals_identity_midsize():
    # a graph too large for a quick oracle run: every set of class m credits
    # its e_m edges, so sum over edges of Y_m = e_m * (sum over vertices of X_m) / k
    from paper_2201_11655_b300 import vdmc
    n, s, d = synth.chung_lu(20000, 5.0, 2.3, 7, reciprocity=0.2)
    with vdmc.graph_create(n, s, d) as g:
        for k in (3, 4):
            x = to_numpy_u64(vdmc.count(g, k)).astype(object).sum(axis=0)
            y = to_numpy_u64(vdmc.count_edges(g, k)).astype(object).sum(axis=0)
            canon = vdmc.class_masks(k)
            nb = k * (k - 1)
            for c, m in enumerate(canon):
                bits = [(int(m) >> (nb - 1 - p)) & 1 for p in range(nb)]
                adj = np.zeros((k, k), int)
                p = 0
                for i in range(k):
                    for j in range(k):
                        if i != j:
                            adj[i, j] = bits[p]
                            p += 1
                e_m = int(((adj + adj.T) > 0).sum()) // 2
                assert y[c] * k == e_m * x[c], (k, c)


def test_variants_relabel_and_direction_invariants_midsize():
    # properties that hold at any size: an undirected count does not depend on
    # arc directions (reversing all arcs, or adding every reverse arc, leaves
    # it unchanged); relabelling the vertices permutes rows (vertex counts)
    # and edge rows (per-edge counts, matched through vdmc_graph_edges)
    from paper_2201_11655_b300 import vdmc
    n, s, d = synth.chung_lu(20000, 5.0, 2.3, 11, reciprocity=0.2)
    vdmc.set_schedule(hub_min_l=16)
    with vdmc.graph_create(n, s, d, undirected=True) as g:
        base = to_numpy_u64(vdmc.count(g, 4))
    with vdmc.graph_create(n, d, s, undirected=True) as g:
        np.testing.assert_array_equal(to_numpy_u64(vdmc.count(g, 4)), base)
    with vdmc.graph_create(n, np.concatenate([s, d]), np.concatenate([d, s]), undirected=True) as g:
        np.testing.assert_array_equal(to_numpy_u64(vdmc.count(g, 4)), base)
    perm = np.random.default_rng(3).permutation(n).astype(np.int32)
    with vdmc.graph_create(n, perm[s], perm[d], undirected=True) as g:
        np.testing.assert_array_equal(to_numpy_u64(vdmc.count(g, 4))[perm], base)
    # per-edge (directed), k=3: relabelled edge rows match
    m, s2, d2 = synth.chung_lu(5000, 4.0, 2.4, 12, reciprocity=0.3)
    with vdmc.graph_create(m, s2, d2) as g:
        u, v, _ = g.edges()
        e0 = to_numpy_u64(vdmc.count_edges(g, 3))
    perm = np.random.default_rng(4).permutation(m).astype(np.int32)
    with vdmc.graph_create(m, perm[s2], perm[d2]) as g:
        u2, v2, _ = g.edges()
        e1 = to_numpy_u64(vdmc.count_edges(g, 3))
    row = {(int(a), int(b)): i for i, (a, b) in enumerate(zip(u2, v2))}
    idx = np.array([row[(min(int(perm[a]), int(perm[b])), max(int(perm[a]), int(perm[b])))] for a, b in zip(u, v)])
    np.testing.assert_array_equal(e1[idx], e0)
