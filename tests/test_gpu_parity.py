"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Every comparison is element by element and bit-exact (uint64 counts; the
output is a unique integer array, so the tolerance is zero).
"""
import math

import numpy as np
import pytest

from conftest import read_golden
from gpu_util import gpu_count, gpu_count_roots, to_numpy_u64
from oracle import oracle as O
from paper_2201_11655_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_11655_b300 import build, vdmc
    build.build()
    vdmc.load()
    torch.cuda.init()


def _arcs(pairs):
    pairs = list(pairs)
    return (np.array([p[0] for p in pairs], np.int32).reshape(-1),
            np.array([p[1] for p in pairs], np.int32).reshape(-1))


def check(n, s, d, ks=(3, 4)):
    for k in ks:
        want, _ = O.count(n, s, d, k)
        got = gpu_count(n, s, d, k)
        np.testing.assert_array_equal(got, want, err_msg="k=%d n=%d m=%d" % (k, n, len(s)))


# ------------------------------------------------------------ graph build --

def test_csr_example_build():
    from paper_2201_11655_b300 import vdmc
    g = read_golden("csr_example.txt")
    arcs = [tuple(int(x) for x in a.split(">")) for a in g["arcs"]]
    s, d = _arcs(arcs)
    with vdmc.graph_create(4, s, d) as G:
        info = G.info()
        rowptr, col, new2old = G.export_csr()
    ui = [int(x) for x in g["undirected_indices"]]
    un = [int(x) for x in g["undirected_neighbors"]]
    di = [int(x) for x in g["directed_indices"]]
    dn = [int(x) for x in g["directed_neighbors"]]
    assert info["edges_u"] == len(un) // 2 and info["arcs_kept"] == len(dn)
    assert info["reciprocal_pairs"] == 1
    # back to original ids: undirected neighbour sets and directed out-lists
    und = {v: set() for v in range(4)}
    out = {v: set() for v in range(4)}
    for r in range(4):
        v = int(new2old[r])
        for e in col[rowptr[r]:rowptr[r + 1]]:
            u = int(new2old[int(e) >> 2])
            und[v].add(u)
            if e & 1:
                out[v].add(u)
    for v in range(4):
        assert sorted(und[v]) == un[ui[v]:ui[v + 1]]
        assert sorted(out[v]) == dn[di[v]:di[v + 1]]
    # rows in rank order are sorted; ranks follow degree descending, id ascending
    deg = np.diff(ui)
    order = np.lexsort((np.arange(4), -deg))
    np.testing.assert_array_equal(new2old, order)


def test_build_counters_and_drops():
    from paper_2201_11655_b300 import vdmc
    n, s, d = synth.gnp(50, 0.1, 3)
    s2 = np.concatenate([s, s[:17], [4, 9, 9]]).astype(np.int32)
    d2 = np.concatenate([d, d[:17], [4, 9, 9]]).astype(np.int32)
    with vdmc.graph_create(n, s2, d2) as G:
        info = G.info()
    assert info["self_loops"] == 3 and info["duplicate_arcs"] == 17
    assert info["arcs_kept"] == len(s)
    pairs = set(zip(s.tolist(), d.tolist()))
    und = {(min(a, b), max(a, b)) for a, b in pairs}
    assert info["edges_u"] == len(und)
    assert info["reciprocal_pairs"] == sum(1 for a, b in pairs if (b, a) in pairs) // 2


def test_build_from_device_pointers():
    n, s, d = synth.chung_lu(500, 3.0, 2.3, 4, reciprocity=0.2)
    want, _ = O.count(n, s, d, 3)
    got = gpu_count(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), 3)
    np.testing.assert_array_equal(got, want)


# ----------------------------------------------------------- hand-worked --

def test_gnp100_full_parity():
    n, s, d = synth.gnp(100, 0.08, 0)
    check(n, s, d)


@pytest.mark.parametrize("n", [4, 5, 9])
def test_complete_digraph(n):
    s, d = _arcs((i, j) for i in range(n) for j in range(n) if i != j)
    check(n, s, d)
    got = gpu_count(n, s, d, 4)
    assert (got[:, 198] == math.comb(n - 1, 3)).all()


def test_cycles_stars_tournament():
    for n in (3, 4, 5, 11):
        s, d = _arcs((i, (i + 1) % n) for i in range(n))
        check(n, s, d)
    for L in (2, 3, 40):
        s, d = _arcs((0, i) for i in range(1, L + 1))
        check(L + 1, s, d)
        check(L + 1, d, s)
    s, d = _arcs((i, j) for i in range(7) for j in range(i + 1, 7))
    check(7, s, d)


# ----------------------------------------------------------- random cases --

@pytest.mark.parametrize("seed", range(12))
def test_random_small(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 300))
    if seed % 2:
        n, s, d = synth.gnp(n, float(rng.uniform(0.01, 0.3)), seed)
    else:
        n, s, d = synth.chung_lu(n, float(rng.uniform(1.0, 6.0)), float(rng.uniform(2.1, 2.8)), seed,
                                 reciprocity=float(rng.uniform(0, 0.5)))
    check(n, s, d)


def test_medium_powerlaw_many_tiles():
    # hubs of a few hundred neighbours: several warps' worth of tasks per root,
    # ragged tails in every inner loop
    n, s, d = synth.chung_lu(3000, 4.0, 2.2, 17, reciprocity=0.2)
    check(n, s, d)


def test_schedules_do_not_change_results():
    from paper_2201_11655_b300 import vdmc
    n, s, d = synth.chung_lu(1500, 4.0, 2.3, 5, reciprocity=0.2)
    want = {k: O.count(n, s, d, k)[0] for k in (3, 4)}
    old = vdmc.get_schedule()
    try:
        for a_chunk, warps, bps, hub, hbps in ((1, 8, 0, 0, 1), (7, 4, 1, 0, 1), (64, 1, 0, 3, 2),
                                               (1000, 2, 3, 1, 1), (16, 8, 0, 20, 3)):
            vdmc.set_schedule(a_chunk=a_chunk, warps_per_block=warps, blocks_per_sm=bps, hub_min_l=hub,
                              hub_blocks_per_sm=hbps)
            for k in (3, 4):
                np.testing.assert_array_equal(gpu_count(n, s, d, k), want[k])
    finally:
        vdmc.set_schedule(**old)



def _full_table_graph(seed):
    """A root r with exactly 64 higher-rank neighbours (the most the warp kernel
    stages) and, among them, a with 128 neighbours of higher rank than r, none
    in N+(r), and a2 with 120 outside N+(r) and 8 inside: the flattened k = 4
    walk's membership table then holds 192 and 184 keys in its 256 slots.
    66 hubs of larger degree (131 private leaves each) take r's lower ranks."""
    rng = np.random.default_rng(seed)
    r, P = 0, list(range(1, 65))
    a, a2 = 1, 2
    nxt = 65
    A = list(range(nxt, nxt + 128)); nxt += 128
    A2 = list(range(nxt, nxt + 120)); nxt += 120
    hubs = list(range(nxt, nxt + 66)); nxt += 66
    edges = [(r, x) for x in P] + [(r, h) for h in hubs] + [(a, y) for y in A] + [(a2, y) for y in A2]
    edges += [(a2, x) for x in P[10:18]]
    for h in hubs:
        edges += [(h, nxt + i) for i in range(131)]
        nxt += 131
    # short paths among the depth-1 and depth-2 vertices (degrees stay far below r's 130)
    for _ in range(150):
        u, v = rng.choice(P[2:] + A + A2, 2, replace=False)
        edges.append((int(u), int(v)))
    src, dst = [], []
    for u, v in edges:
        if u == v:
            continue
        if rng.random() < 0.5:
            u, v = v, u
        src.append(u); dst.append(v)
        if rng.random() < 0.2:
            src.append(v); dst.append(u)
    return nxt, np.array(src, np.int32), np.array(dst, np.int32)


@pytest.mark.parametrize("seed", [0, 1])
def test_warp_kernel_membership_table_at_capacity(seed):
    from paper_2201_11655_b300 import vdmc
    n, s, d = _full_table_graph(seed)
    with vdmc.graph_create(n, s, d) as g:
        rowptr, col, new2old = g.export_csr()
    old2new = np.empty(n, np.int64)
    old2new[new2old] = np.arange(n)
    rr = int(old2new[0])
    ranks = (col[rowptr[rr]:rowptr[rr + 1]] >> 2).astype(np.int64)
    assert int((ranks > rr).sum()) == 64            # N+(r): the staging limit
    for v in (1, 2):                                # a, a2: 128 neighbours above r
        rv = int(old2new[v])
        rk = (col[rowptr[rv]:rowptr[rv + 1]] >> 2).astype(np.int64)
        assert rv > rr and int((rk > rr).sum()) == 128
    old = vdmc.get_schedule()
    try:
        vdmc.set_schedule(hub_min_l=0)              # every root through the warp kernel
        check(n, s, d)
    finally:
        vdmc.set_schedule(**old)


_SPLIT_GRAPH = {}


@pytest.mark.parametrize("warps", [16, 32])
@pytest.mark.parametrize("split,roots,hub", [(1, 0, 8), (2, 5, 8), (3, 1000, 4), (4, 7, 1), (16, 3, 16), (5, 40, 2)])
def test_split_roots_match_oracle(split, roots, hub, warps):
    # the largest roots counted by several CTAs (members and second-hop
    # vertices shared out, three-member partials summed before the division),
    # with 16- and 32-warp CTAs
    from paper_2201_11655_b300 import vdmc
    if not _SPLIT_GRAPH:
        n, s, d = synth.chung_lu(1500, 4.0, 2.3, 5, reciprocity=0.2)
        _SPLIT_GRAPH.update(n=n, s=s, d=d, want={k: O.count(n, s, d, k)[0] for k in (3, 4)})
    n, s, d, want = _SPLIT_GRAPH["n"], _SPLIT_GRAPH["s"], _SPLIT_GRAPH["d"], _SPLIT_GRAPH["want"]
    old = vdmc.get_schedule()
    try:
        vdmc.set_schedule(hub_min_l=hub, hub_split=split, hub_split_roots=roots, hub_warps=warps)
        for k in (3, 4):
            np.testing.assert_array_equal(gpu_count(n, s, d, k), want[k], err_msg="k=%d" % k)
    finally:
        vdmc.set_schedule(**old)


def test_split_roots_with_rank_ranges():
    # a root range that cuts through the split roots: every part of a root in
    # range counts, every part of a root out of range skips
    from paper_2201_11655_b300 import vdmc
    n, s, d = synth.chung_lu(800, 5.0, 2.2, 9, reciprocity=0.3)
    old = vdmc.get_schedule()
    try:
        vdmc.set_schedule(hub_min_l=0)
        whole = gpu_count(n, s, d, 4)
        vdmc.set_schedule(hub_min_l=4, hub_split=3, hub_split_roots=10)
        with vdmc.graph_create(n, s, d) as g:
            acc = torch.zeros((n, 199), dtype=torch.int64, device="cuda")
            for lo, hi in ((0, 2), (2, 7), (7, 30), (30, n)):
                part = vdmc.count_roots(g, 4, lo, hi)
                acc += part.view(torch.int64)
            torch.cuda.synchronize()
            assert g.device_status() == 0
        np.testing.assert_array_equal(acc.cpu().numpy().view(np.uint64), whole)
    finally:
        vdmc.set_schedule(**old)


@pytest.fixture
def schedule():
    from paper_2201_11655_b300 import vdmc
    old = vdmc.get_schedule()
    yield vdmc
    vdmc.set_schedule(**old)


@pytest.mark.parametrize("hub_min_l", [0, 1])
@pytest.mark.parametrize("seed", range(10))
def test_root_per_cta_kernel_vs_oracle(schedule, hub_min_l, seed):
    # hub_min_l = 1 sends every root to the root-per-CTA (signature counting)
    # kernel, 0 every root to the warp-per-task (plain enumeration) kernel.
    schedule.set_schedule(hub_min_l=hub_min_l)
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(4, 250))
    kind = seed % 3
    if kind == 0:
        n, s, d = synth.gnp(n, float(rng.uniform(0.02, 0.4)), seed)
    elif kind == 1:
        n, s, d = synth.chung_lu(n, float(rng.uniform(1.0, 8.0)), float(rng.uniform(2.05, 2.6)), seed,
                                 reciprocity=float(rng.uniform(0, 0.6)))
    else:
        # dense core + sparse periphery: many H-edges, wedges and triangles
        n1, s1, d1 = synth.gnp(min(n, 30), 0.5, seed)
        n2, s2, d2 = synth.chung_lu(n, 3.0, 2.2, seed + 1, reciprocity=0.3)
        s, d = np.concatenate([s1, s2]), np.concatenate([d1, d2])
    check(n, s, d)


def test_root_per_cta_kernel_medium_powerlaw(schedule):
    n, s, d = synth.chung_lu(4000, 5.0, 2.1, 31, reciprocity=0.25)
    for hub in (1, 16, 200):
        schedule.set_schedule(hub_min_l=hub)
        check(n, s, d)


# ---------------------------------------------------------------- edges --

def test_empty_and_degenerate():
    from paper_2201_11655_b300 import vdmc
    e = np.zeros(0, np.int32)
    for n in (0, 1, 6):
        for k in (3, 4):
            got = gpu_count(n, e, e, k)
            assert got.shape == (n, vdmc.num_classes(k)) and not got.any()
    # only self-loops
    s = np.arange(5, dtype=np.int32)
    assert not gpu_count(5, s, s, 4).any()
    # a single arc: no 3-set is connected
    assert not gpu_count(2, np.array([0], np.int32), np.array([1], np.int32), 3).any()
    # fewer vertices than k
    check(3, *_arcs([(0, 1), (1, 2), (2, 0)]), ks=(4,))


def test_errors():
    from paper_2201_11655_b300 import vdmc
    with pytest.raises(vdmc.VdmcError) as ei:
        vdmc.graph_create(5, np.array([0, 5], np.int32), np.array([1, 2], np.int32))
    assert ei.value.status == 2
    with pytest.raises(vdmc.VdmcError) as ei:
        vdmc.graph_create(5, np.array([0, -1], np.int32), np.array([1, 2], np.int32))
    assert ei.value.status == 2
    n, s, d = synth.gnp(10, 0.3, 1)
    with vdmc.graph_create(n, s, d) as g:
        with pytest.raises(ValueError):
            vdmc.count(g, 5)
        import ctypes
        out = torch.zeros(n * 13, dtype=torch.uint64, device="cuda")
        st = vdmc.load().vdmc_count(g.handle, 5, ctypes.c_void_p(out.data_ptr()), None)
        assert st == 1


# ------------------------------------------------------------ root ranges --

def test_root_ranges_partition_and_match_oracle():
    from paper_2201_11655_b300 import vdmc
    n, s, d = synth.chung_lu(2000, 4.0, 2.3, 23, reciprocity=0.2)
    rank = O.degree_rank(n, s, d)
    with vdmc.graph_create(n, s, d) as g:
        _, _, new2old = g.export_csr()
        np.testing.assert_array_equal(rank[new2old], np.arange(n))
        for k in (3, 4):
            acc = np.zeros((n, vdmc.num_classes(k)), np.uint64)
            for lo, hi in ((0, 1), (1, 17), (17, 400), (400, n)):
                part = gpu_count_roots(g, k, lo, hi)
                want, _ = O.count_roots(n, s, d, k, rank, lo, hi)
                np.testing.assert_array_equal(part, want)
                acc += part
            full = to_numpy_u64(vdmc.count(g, k))
            np.testing.assert_array_equal(acc, full)


def test_repeated_calls_overwrite():
    from paper_2201_11655_b300 import vdmc
    n, s, d = synth.gnp(120, 0.06, 9)
    want, _ = O.count(n, s, d, 4)
    with vdmc.graph_create(n, s, d) as g:
        out = torch.full((n, 199), 7, dtype=torch.uint64, device="cuda")
        for _ in range(3):
            vdmc.count(g, 4, out=out)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(to_numpy_u64(out), want)
