"""GPU checks of the measurement hooks and of root-range sharding on one GPU.

* vdmc_work_model's entry counts equal the same sums written out in numpy
  over the exported CSR (N(r), N(a) per depth-1 vertex, N(b) per distinct
  depth-2 vertex and per (a, b) use);
* vdmc_count_stats splits every count exactly: sets enumerated one by one
  plus sets accounted for by signature = the count's number of sets, under
  several schedules;
* the equal-work partition of the rank space (vdmc_root_costs + the host
  cut) gives ranges whose counts sum to the full count bit for bit (Lemma 1),
  which is what each GPU of a sharded count contributes.
"""
import numpy as np
import pytest

from gpu_util import to_numpy_u64
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
    old = vdmc.get_schedule()
    yield
    vdmc.set_schedule(**old)


def model_by_definition(rowptr, col, k):
    n = rowptr.size - 1
    nb = [(col[rowptr[r]:rowptr[r + 1]] >> 2).astype(np.int64) for r in range(n)]
    deg = np.diff(rowptr)
    er = ea = ed = eu = 0
    for r in range(n):
        P = nb[r][nb[r] > r]
        er += deg[r]
        ea += int(deg[P].sum())
        if k == 4:
            Nr = set(nb[r].tolist())
            seen = set()
            for a in P:
                for b in nb[a]:
                    if b > r and b not in Nr:
                        eu += int(deg[b])
                        if b not in seen:
                            seen.add(b)
                            ed += int(deg[b])
    return er, ea, ed, eu


@pytest.mark.parametrize("k", [3, 4])
def test_work_model_matches_definition(k):
    from paper_2201_11655_b300 import vdmc
    for n, s, d in (synth.gnp(60, 0.1, 1), synth.chung_lu(800, 3.0, 2.3, 5, reciprocity=0.2)):
        with vdmc.graph_create(n, s, d) as g:
            m = g.work_model(k)
            rowptr, col, _ = g.export_csr()
        er, ea, ed, eu = model_by_definition(rowptr, col, k)
        assert (m["entries_root"], m["entries_depth1"]) == (er, ea)
        assert (m["entries_depth2"], m["entries_depth2_per_use"]) == ((ed, eu) if k == 4 else (0, 0))
        C = vdmc.num_classes(k)
        assert m["output_bytes"] == 8 * n * C + 4 * n
        assert m["bytes"] == 4 * (er + ea + ed) + m["output_bytes"]
        assert m["bytes_per_use"] == 4 * (er + ea + eu) + m["output_bytes"]


@pytest.mark.parametrize("sched", [dict(hub_min_l=0), dict(hub_min_l=1), dict(hub_min_l=8, hub_split=3, hub_split_roots=4),
                                   dict(hub_min_l=16, hub_warps=32)])
def test_count_stats_split_every_set(sched):
    from paper_2201_11655_b300 import vdmc
    n, s, d = synth.chung_lu(3000, 4.0, 2.2, 41, reciprocity=0.2)
    vdmc.set_schedule(**sched)
    with vdmc.graph_create(n, s, d) as g:
        for k in (3, 4):
            out = vdmc.count(g, k)
            torch.cuda.synchronize()
            sets = int(out.view(torch.int64).sum().item()) // k
            st = g.count_stats()
            assert st["sets_enumerated"] + st["sets_by_signature"] == sets
            assert st["sets_plain"] + st["sets_hub"] == sets
            if sched["hub_min_l"] == 0:
                assert st["sets_hub"] == 0 and st["sets_by_signature"] == 0
            else:
                assert st["sets_hub"] > 0 and st["sets_by_signature"] > 0


@pytest.mark.parametrize("parts", [2, 3, 8])
def test_equal_work_partition_sums_to_full_count(parts):
    from paper_2201_11655_b300 import shard, vdmc
    n, s, d = synth.chung_lu(20000, 5.0, 2.3, 7, reciprocity=0.2)
    vdmc.set_schedule(hub_min_l=16, hub_split=2, hub_split_roots=8)
    with vdmc.graph_create(n, s, d) as g:
        for k in (3, 4):
            full = to_numpy_u64(vdmc.count(g, k))
            costs = shard.root_costs(g, k)
            assert costs.size == n and int(costs.sum()) > 0
            bounds = shard.partition(g, k, parts)
            assert bounds[0] == 0 and bounds[-1] == n and len(bounds) == parts + 1
            acc = np.zeros_like(full)
            for i in range(parts):
                acc += to_numpy_u64(vdmc.count_roots(g, k, bounds[i], bounds[i + 1]))
            torch.cuda.synchronize()
            assert g.device_status() == 0
            np.testing.assert_array_equal(acc, full)
