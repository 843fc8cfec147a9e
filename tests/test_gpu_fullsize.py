"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

The oracle cannot count the full graphs, so it checks sampled root ranges
(every set whose lowest-rank member lies in the range, by Lemma 1) across the
degree spectrum; the rest is checked by properties that hold at any size:
ranges partition the full count, the two counting kernels agree on heavy
roots, and the k=3 totals obey the degree/triangle identity.
"""
import math
import os

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


def check_range(vdmc, g, n, s, d, k, rank, lo, hi):
    out = vdmc.count_roots(g, k, lo, hi)
    torch.cuda.synchronize()
    assert g.device_status() == 0
    ids, rows, total = rows_of(out)
    want, found = O.count_roots(n, s, d, k, rank, lo, hi)
    wids = np.nonzero(want.sum(axis=1))[0]
    np.testing.assert_array_equal(ids, wids, err_msg="k=%d ranks [%d,%d)" % (k, lo, hi))
    np.testing.assert_array_equal(rows, want[wids], err_msg="k=%d ranks [%d,%d)" % (k, lo, hi))
    assert total == k * found
    return found


@pytest.fixture(scope="module")
def powerlaw(env):
    vdmc, autotune = env
    n, s, d = synth.workload("chunglu_n1M_m10M_a2.3_r0.2")
    autotune.apply_tuned(4, n, len(s))
    g = vdmc.graph_create(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda())
    rank = O.degree_rank(n, s, d)
    yield vdmc, g, n, s, d, rank
    g.close()


def test_powerlaw_root_samples_vs_oracle(powerlaw):
    vdmc, g, n, s, d, rank = powerlaw
    info = g.info()
    assert info["num_hub_roots"] > 0
    # Root samples across the degree spectrum, each small enough for the
    # oracle (it runs one root per thread; the heaviest roots hold ~10^12
    # 4-sets and are checked below by kernel agreement and partitions).
    for lo, hi in ((5000, 5100), (60_000, 61_000), (700_000, 720_000)):
        check_range(vdmc, g, n, s, d, 3, rank, lo, hi)
    # k=4: roots of the root-per-CTA kernel (L >= 32 under the tuned
    # schedule) and of the warp-per-task kernel
    for lo, hi in ((8000, 8010), (20_000, 20_100), (200_000, 203_000)):
        check_range(vdmc, g, n, s, d, 4, rank, lo, hi)


def test_powerlaw_partition_and_kernel_agreement(powerlaw):
    vdmc, g, n, s, d, rank = powerlaw
    full = vdmc.count(g, 4)
    acc = torch.zeros_like(full.view(torch.int64))
    for lo, hi in ((0, 30), (30, 5000), (5000, n)):
        acc += vdmc.count_roots(g, 4, lo, hi).view(torch.int64)
    torch.cuda.synchronize()
    assert torch.equal(acc, full.view(torch.int64))
    # heavy roots through each kernel
    old = vdmc.get_schedule()
    try:
        vdmc.set_schedule(hub_min_l=1)
        a = vdmc.count_roots(g, 4, 2000, 2003).view(torch.int64).clone()
        vdmc.set_schedule(hub_min_l=0)
        b = vdmc.count_roots(g, 4, 2000, 2003).view(torch.int64).clone()
        torch.cuda.synchronize()
        assert int(a.sum()) > 0 and torch.equal(a, b)
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


def test_er4m_root_samples_vs_oracle(env):
    vdmc, autotune = env
    n, s, d = synth.workload("er_n4M_m32M")
    g = vdmc.graph_create(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda())
    rank = O.degree_rank(n, s, d)
    try:
        check_range(vdmc, g, n, s, d, 4, rank, 0, 400)
        full = vdmc.count(g, 4).view(torch.int64)
        part = vdmc.count_roots(g, 4, 0, 1_000_000).view(torch.int64) + \
            vdmc.count_roots(g, 4, 1_000_000, n).view(torch.int64)
        torch.cuda.synchronize()
        assert torch.equal(full, part)
    finally:
        g.close()
