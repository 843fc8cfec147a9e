"""Serving loop on the GPU: every result is the same alone and in the mix.

A stream of small and medium requests (k = 3 and 4) is served with
continuous batching; each request's counts must equal the same graph counted
alone (and the oracle for the small ones) bit for bit -- the output is an
exact integer array, so the tolerance is zero.
"""
import numpy as np
import pytest

from gpu_util import gpu_count, to_numpy_u64
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


@pytest.mark.parametrize("workers", [4, 0])
def test_served_equals_alone(workers):
    from paper_2201_11655_b300.serve import GpuBackend, Request, Server
    rng = np.random.default_rng(3)
    reqs = []
    for i in range(60):
        if i % 10 == 9:
            n, s, d = synth.chung_lu(int(rng.integers(5000, 20000)), float(rng.uniform(4, 10)), 2.3,
                                     1000 + i, reciprocity=0.2)
        elif i % 2:
            n, s, d = synth.gnp(int(rng.integers(20, 200)), float(rng.uniform(0.02, 0.15)), 1000 + i)
        else:
            n, s, d = synth.chung_lu(int(rng.integers(30, 300)), float(rng.uniform(1.5, 5)), 2.5, 1000 + i)
        reqs.append(Request(rid=i, n=n, src=s, dst=d, k=3 + (i % 3 == 0), arrival=i * 2e-4))
    backend = GpuBackend(workers=workers)
    srv = Server(backend, memory_budget=8 << 30, max_inflight=4, small_n=2000, batch_max=16, batch_wait=1e-3)
    srv.submit_stream(reqs)
    done = srv.run()
    torch.cuda.synchronize()
    assert len(done) == len(reqs) and all(r.error is None for r in done)
    assert any(len([x for x in done if x.job == r.job]) > 1 for r in done)  # some batches formed
    for r in done:
        got = to_numpy_u64(r.counts.contiguous())
        alone = gpu_count(r.n, r.src, r.dst, r.k)
        np.testing.assert_array_equal(got, alone, err_msg="request %d" % r.rid)
        if r.n <= 300:
            want, _ = O.count(r.n, r.src, r.dst, r.k)
            np.testing.assert_array_equal(got, want)
    st = Server.latency_stats(done)
    assert st["count"] == len(reqs) and st["p99_ms"] >= st["p50_ms"]
    backend.close()


def test_threads_counting_different_graphs_concurrently():
    # host threads build and count graphs of different sizes at the same time
    # (as the serving backend's workers do); each result equals the graph
    # counted alone
    import concurrent.futures
    from paper_2201_11655_b300 import vdmc
    old = vdmc.get_schedule()
    vdmc.set_schedule(hub_min_l=8)
    try:
        graphs = [synth.chung_lu(int(n), 4.0, 2.2, 50 + i, reciprocity=0.2)
                  for i, n in enumerate((300, 3000, 20000, 800, 60000, 1500, 9000, 40000))]
        alone = [gpu_count(n, s, d, 4) for n, s, d in graphs]

        def work(i):
            torch.cuda.set_device(0)
            n, s, d = graphs[i]
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                with vdmc.graph_create(n, s, d, stream=stream) as g:
                    out = vdmc.count(g, 4, stream=stream)
                    stream.synchronize()
                    assert g.device_status() == 0
                    return to_numpy_u64(out)

        for rep in range(3):
            with concurrent.futures.ThreadPoolExecutor(max_workers=4) as ex:
                got = list(ex.map(work, range(len(graphs))))
            for i in range(len(graphs)):
                np.testing.assert_array_equal(got[i], alone[i], err_msg="graph %d rep %d" % (i, rep))
    finally:
        vdmc.set_schedule(**old)
