"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

The oracle cannot count the full graphs, so it checks sampled root ranges
(every set whose lowest-rank member lies in the range, by Lemma 1): the
heaviest roots at k=3, a heavy root of the root-per-CTA kernel at k=4, and
ranges stratified over the degree deciles.  The rest is checked by properties
that hold at any size:
  * transposing every arc permutes the classes (the class-transpose map is
    taken from the oracle's canonical index), so count(G^T) must equal
    count(G) with its columns permuted -- every hub root is counted again with
    its colours swapped;
  * relabelling the vertices permutes the rows (and reorders equal-degree
    roots, so different roots take different kernel paths);
  * disjoint rank ranges sum to the full count;
  * the two counting kernels agree on split and unsplit heavy roots;
  * the k=3 totals obey the degree/triangle identity.
Range sizes are chosen by probing the set count on the device (a size, not an
expected value); every expected value comes from the oracle or from the
untransformed count.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2201_11655_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_11655_b300 import autotune, build, vdmc
    build.build()
    vdmc.load()
    old = vdmc.get_schedule()
    yield vdmc, autotune
    vdmc.set_schedule(**old)


def rows_of(out):
    """(row ids, rows) of the non-zero rows of a device count array, plus its total."""
    o = out.view(torch.int64)
    nz = torch.nonzero(o.sum(dim=1)).flatten()
    return nz.cpu().numpy(), o[nz].cpu().numpy().view(np.uint64), int(o.sum().item())


def compare_rows(got, want, k, found, what):
    ids, rows, total = rows_of(got)
    wids = np.nonzero(want.sum(axis=1))[0]
    np.testing.assert_array_equal(ids, wids, err_msg="k=%d %s: non-zero rows" % (k, what))
    np.testing.assert_array_equal(rows, want[wids], err_msg="k=%d %s" % (k, what))
    assert total == k * found


def check_range(vdmc, g, n, s, d, k, rank, lo, hi):
    out = vdmc.count_roots(g, k, lo, hi)
    torch.cuda.synchronize()
    assert g.device_status() == 0
    want, found = O.count_roots(n, s, d, k, rank, lo, hi)
    compare_rows(out, want, k, found, "ranks [%d,%d)" % (lo, hi))
    return found


def check_ranges(vdmc, g, n, s, d, k, rank, ranges):
    """Many disjoint rank ranges against one oracle call over all of them."""
    acc = None
    for lo, hi in ranges:
        part = vdmc.count_roots(g, k, lo, hi).view(torch.int64)
        acc = part.clone() if acc is None else acc.add_(part)
    torch.cuda.synchronize()
    assert g.device_status() == 0
    want, found = O.count_root_ranges(n, s, d, k, rank, ranges)
    compare_rows(acc, want, k, found, "%d ranges" % len(ranges))
    return found


def sets_in(vdmc, g, k, lo, hi):
    out = vdmc.count_roots(g, k, lo, hi)
    return int(out.view(torch.int64).sum().item()) // k


def stratified_ranges(vdmc, g, k, n, per_decile, budget, skip_heavy=0):
    """per_decile ranges in each tenth of the rank space, each grown (by
    doubling from one root) while its set count stays within budget; a start
    whose single root exceeds the budget moves to a lighter rank."""
    ranges = []
    for dec in range(10):
        for i in range(per_decile):
            lo = dec * n // 10 + i * n // (10 * per_decile)
            lo = max(lo, skip_heavy)
            while lo < n - 1 and sets_in(vdmc, g, k, lo, lo + 1) > budget:
                lo = lo * 2 + 1
            if lo >= n:
                continue
            w = 1
            while lo + 2 * w <= n and w < 4096 and sets_in(vdmc, g, k, lo, lo + 2 * w) <= budget:
                w *= 2
            if not ranges or lo >= ranges[-1][1]:
                ranges.append((lo, min(n, lo + w)))
    return ranges


def class_transpose_map(k):
    """tau[c] = column of the class of the transposed motif of column c (oracle tables)."""
    canon, _ = O.classes(k)
    col = {int(m): i for i, m in enumerate(canon)}
    nb = k * (k - 1)
    tau = []
    for m in canon:
        bits = [(int(m) >> (nb - 1 - p)) & 1 for p in range(nb)]
        adj = np.zeros((k, k), int)
        p = 0
        for i in range(k):
            for j in range(k):
                if i != j:
                    adj[i, j] = bits[p]
                    p += 1
        t = adj.T
        idx = 0
        for i in range(k):
            for j in range(k):
                if i != j:
                    idx = (idx << 1) | int(t[i, j])
        tau.append(col[O.canonical_index(k, idx)])
    return np.array(tau)


def check_transpose(vdmc, n, s, d, k, out):
    """count(G^T)[:, tau[c]] == count(G)[:, c] for every column c."""
    tau = torch.from_numpy(class_transpose_map(k)).cuda()
    with vdmc.graph_create(n, torch.from_numpy(d).cuda(), torch.from_numpy(s).cuda()) as gt:
        ot = vdmc.count(gt, k).view(torch.int64)
        torch.cuda.synchronize()
        assert gt.device_status() == 0
        assert torch.equal(ot[:, tau], out.view(torch.int64)), "k=%d transpose" % k


def check_relabel(vdmc, n, s, d, k, out, seed):
    """count(pi(G))[pi(v)] == count(G)[v] for a random relabelling pi."""
    perm = np.random.default_rng(seed).permutation(n).astype(np.int32)
    ps = torch.from_numpy(perm[s]).cuda()
    pd = torch.from_numpy(perm[d]).cuda()
    with vdmc.graph_create(n, ps, pd) as gp:
        op = vdmc.count(gp, k).view(torch.int64)
        torch.cuda.synchronize()
        assert gp.device_status() == 0
        assert torch.equal(op[torch.from_numpy(perm).long().cuda()], out.view(torch.int64)), "k=%d relabel" % k


@pytest.fixture(scope="module")
def powerlaw(env):
    vdmc, autotune = env
    n, s, d = synth.workload("chunglu_n1M_m10M_a2.3_r0.2")
    autotune.apply_tuned(4, n, len(s))
    g = vdmc.graph_create(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda())
    rank = O.degree_rank(n, s, d)
    yield vdmc, g, n, s, d, rank
    g.close()


def test_powerlaw_heaviest_roots_k3_vs_oracle(powerlaw):
    # rank 0 (17,018 higher-rank neighbours, ~1.5e8 sets) and ranks 31, 32:
    # the last split root and the first unsplit root of the tuned schedule
    vdmc, g, n, s, d, rank = powerlaw
    assert g.info()["num_hub_roots"] > 0
    assert vdmc.get_schedule()["hub_split_roots"] >= 32
    check_range(vdmc, g, n, s, d, 3, rank, 0, 1)
    check_range(vdmc, g, n, s, d, 3, rank, 31, 33)


def test_powerlaw_hub_root_k4_vs_oracle(powerlaw):
    # rank 1000: 640 higher-rank neighbours, ~7e7 sets, root-per-CTA kernel
    vdmc, g, n, s, d, rank = powerlaw
    check_range(vdmc, g, n, s, d, 4, rank, 1000, 1001)


@pytest.mark.parametrize("k,budget", [(3, 2_000_000), (4, 2_000_000)])
def test_powerlaw_stratified_ranges_vs_oracle(powerlaw, k, budget):
    vdmc, g, n, s, d, rank = powerlaw
    ranges = stratified_ranges(vdmc, g, k, n, per_decile=5, budget=budget, skip_heavy=2000 if k == 4 else 0)
    assert len(ranges) >= 50
    check_ranges(vdmc, g, n, s, d, k, rank, ranges)


@pytest.mark.parametrize("k", [3, 4])
def test_powerlaw_transpose_and_relabel(powerlaw, k):
    vdmc, g, n, s, d, rank = powerlaw
    out = vdmc.count(g, k)
    torch.cuda.synchronize()
    assert g.device_status() == 0
    check_transpose(vdmc, n, s, d, k, out)
    check_relabel(vdmc, n, s, d, k, out, seed=11 + k)


def test_powerlaw_partition_and_kernel_agreement(powerlaw):
    vdmc, g, n, s, d, rank = powerlaw
    full = vdmc.count(g, 4)
    acc = torch.zeros_like(full.view(torch.int64))
    for lo, hi in ((0, 30), (30, 5000), (5000, n)):
        acc += vdmc.count_roots(g, 4, lo, hi).view(torch.int64)
    torch.cuda.synchronize()
    assert torch.equal(acc, full.view(torch.int64))
    # heavy roots through each kernel: rank 31 (a split root under the tuned
    # schedule), rank 32 (the first unsplit one), rank 300
    old = vdmc.get_schedule()
    try:
        for lo, hi in ((31, 32), (32, 33), (300, 301)):
            vdmc.set_schedule(hub_min_l=1)
            a = vdmc.count_roots(g, 4, lo, hi).view(torch.int64).clone()
            vdmc.set_schedule(hub_min_l=0)
            b = vdmc.count_roots(g, 4, lo, hi).view(torch.int64).clone()
            torch.cuda.synchronize()
            assert g.device_status() == 0
            assert int(a.sum()) > 0 and torch.equal(a, b), "ranks [%d,%d)" % (lo, hi)
    finally:
        vdmc.set_schedule(**old)


def test_powerlaw_k3_degree_triangle_identity(powerlaw):
    # connected 3-sets through v = C(d_v, 2) + sum_{a in N(v)} (d_a - 1) - 2 tri(v),
    # with tri(v) the sum of the triangle classes' columns
    vdmc, g, n, s, d, rank = powerlaw
    out = vdmc.count(g, 3).view(torch.int64)
    rowptr, col, new2old = g.export_csr()
    deg_r = np.diff(rowptr)
    nb = (col >> 2).astype(np.int64)
    rows = np.repeat(np.arange(n), deg_r)
    nbsum = np.bincount(rows, weights=(deg_r[nb] - 1).astype(np.float64), minlength=n).astype(np.int64)
    masks = vdmc.class_masks(3)
    tri_cols = [c for c, m in enumerate(masks)
                if all(((int(m) >> (5 - p)) & 1) or ((int(m) >> (5 - q)) & 1) for p, q in ((0, 2), (1, 4), (3, 5)))]
    tot = out.sum(dim=1).cpu().numpy()
    tri = out[:, tri_cols].sum(dim=1).cpu().numpy()
    deg_o = np.empty(n, np.int64)
    deg_o[new2old] = deg_r
    nbs_o = np.empty(n, np.int64)
    nbs_o[new2old] = nbsum
    np.testing.assert_array_equal(tot, deg_o * (deg_o - 1) // 2 + nbs_o - 2 * tri)


@pytest.fixture(scope="module")
def er4m(env):
    vdmc, autotune = env
    n, s, d = synth.workload("er_n4M_m32M")
    autotune.apply_tuned(4, n, len(s))
    g = vdmc.graph_create(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda())
    rank = O.degree_rank(n, s, d)
    yield vdmc, g, n, s, d, rank
    g.close()


def test_er4m_ranges_across_rank_space_vs_oracle(er4m):
    # 25 ranges of 400 roots spread over the whole rank space, plus the
    # highest-degree roots
    vdmc, g, n, s, d, rank = er4m
    ranges = [(0, 400)] + [(j * n // 25, j * n // 25 + 400) for j in range(1, 25)]
    check_ranges(vdmc, g, n, s, d, 4, rank, ranges)


def test_er4m_transpose_relabel_partition(er4m):
    vdmc, g, n, s, d, rank = er4m
    full = vdmc.count(g, 4)
    torch.cuda.synchronize()
    assert g.device_status() == 0
    part = vdmc.count_roots(g, 4, 0, 1_000_000).view(torch.int64) + \
        vdmc.count_roots(g, 4, 1_000_000, n).view(torch.int64)
    torch.cuda.synchronize()
    assert torch.equal(full.view(torch.int64), part)
    check_transpose(vdmc, n, s, d, 4, full)
    check_relabel(vdmc, n, s, d, 4, full, seed=5)
