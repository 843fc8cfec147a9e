"""Host-side logic of the serving loop, on a simulated backend (no GPU).

The backend finishes a job a fixed simulated time after launch; the clock is
advanced by hand, so every scheduling decision is deterministic.
"""
import numpy as np

from paper_2201_11655_b300.serve import Request, Server, footprint_bytes


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeBackend:
    def __init__(self, clock, per_vertex=1e-6, fail_n=None):
        self.clock = clock
        self.per_vertex = per_vertex
        self.fail_n = fail_n
        self.launched = []

    def launch(self, reqs):
        if self.fail_n is not None and any(r.n == self.fail_n for r in reqs):
            raise RuntimeError("simulated launch failure")
        self.launched.append([r.rid for r in reqs])
        return {"t": self.clock() + 1e-3 + self.per_vertex * sum(r.n for r in reqs), "reqs": reqs}

    def done(self, h):
        return self.clock() >= h["t"]

    def finish(self, h):
        return [("counts", r.rid) for r in h["reqs"]]


def mk(rid, n, k, t, m=None):
    m = m if m is not None else 4 * n
    e = np.zeros(m, np.int32)
    return Request(rid=rid, n=n, src=e, dst=e, k=k, arrival=t)


def drive(server, clock, dt=1e-4, limit=10**6):
    steps = 0
    while not server.idle():
        server.poll()
        clock.t += dt
        steps += 1
        assert steps < limit
    return server.completed


def test_all_complete_and_small_requests_are_batched():
    clock = Clock()
    be = FakeBackend(clock)
    srv = Server(be, memory_budget=10 ** 12, max_inflight=2, small_n=1000, batch_max=8, batch_wait=5e-3, clock=clock)
    reqs = [mk(i, 100 + i, 3 + (i % 2), t=i * 1e-4) for i in range(40)] + [mk(100, 50_000, 4, t=1e-3)]
    srv.submit_stream(reqs)
    done = drive(srv, clock)
    assert sorted(r.rid for r in done) == sorted(r.rid for r in reqs)
    assert all(r.counts == ("counts", r.rid) for r in done)
    sizes = [len(j) for j in be.launched]
    assert max(sizes) > 1 and max(sizes) <= 8
    # a batch holds one k only
    by_id = {r.rid: r for r in reqs}
    for j in be.launched:
        assert len({by_id[i].k for i in j}) == 1
    stats = Server.latency_stats(done)
    assert stats["count"] == len(reqs) and stats["p99_ms"] >= stats["p50_ms"] > 0


def test_memory_budget_is_respected():
    clock = Clock()
    be = FakeBackend(clock, per_vertex=1e-5)
    one = footprint_bytes(20_000, 80_000, 4)
    srv = Server(be, memory_budget=int(2.5 * one), max_inflight=8, small_n=100, clock=clock)
    reqs = [mk(i, 20_000, 4, t=0.0) for i in range(7)]
    srv.submit_stream(reqs)
    peak_jobs = 0
    while not srv.idle():
        srv.poll()
        peak_jobs = max(peak_jobs, len(srv.inflight))
        assert srv.reserved <= srv.budget
        clock.t += 1e-4
    assert peak_jobs == 2          # 2.5 requests' worth of memory -> 2 at a time
    assert srv.peak_reserved <= srv.budget
    assert len(srv.completed) == 7


def test_oversize_request_runs_alone():
    clock = Clock()
    be = FakeBackend(clock)
    srv = Server(be, memory_budget=footprint_bytes(1000, 4000, 3), max_inflight=4, small_n=10, clock=clock)
    reqs = [mk(0, 200_000, 4, 0.0), mk(1, 500, 3, 0.0), mk(2, 600, 3, 0.0)]
    srv.submit_stream(reqs)
    done = drive(srv, clock)
    assert len(done) == 3
    first = be.launched[0]
    assert first == [0]             # the big one, alone, when nothing else holds memory


def test_large_requests_fifo_and_inflight_cap():
    clock = Clock()
    be = FakeBackend(clock, per_vertex=1e-6)
    srv = Server(be, memory_budget=10 ** 13, max_inflight=3, small_n=10, clock=clock)
    reqs = [mk(i, 5000 + i, 4, t=0.0) for i in range(10)]
    srv.submit_stream(reqs)
    while not srv.idle():
        srv.poll()
        assert len(srv.inflight) <= 3
        clock.t += 1e-4
    assert [j[0] for j in be.launched] == list(range(10))


def test_failed_launch_reports_error_and_continues():
    clock = Clock()
    be = FakeBackend(clock, fail_n=777)
    srv = Server(be, memory_budget=10 ** 12, max_inflight=2, small_n=10, clock=clock)
    srv.submit_stream([mk(0, 777, 3, 0.0), mk(1, 800, 3, 0.0)])
    done = drive(srv, clock)
    errs = {r.rid: r.error for r in done}
    assert errs[0] and errs[1] is None


class FailingFinishBackend(FakeBackend):
    """finish() raises for jobs holding a request of a given size (a device
    status error, simulated on the host)."""

    def __init__(self, clock, bad_n):
        super().__init__(clock)
        self.bad_n = bad_n

    def finish(self, h):
        if any(r.n == self.bad_n for r in h["reqs"]):
            raise RuntimeError("device status 5")
        return super().finish(h)


def test_failed_job_does_not_stop_the_loop():
    clock = Clock()
    srv = Server(FailingFinishBackend(clock, bad_n=50_000), memory_budget=10 ** 12, max_inflight=2, small_n=1000,
                 batch_max=4, batch_wait=1e-3, clock=clock)
    reqs = [mk(i, 100 + i, 3, t=i * 1e-4) for i in range(12)] + [mk(99, 50_000, 4, t=2e-4)]
    srv.submit_stream(reqs)
    done = drive(srv, clock)
    assert len(done) == len(reqs)
    bad = [r for r in done if r.error]
    assert [r.rid for r in bad] == [99] and "status" in bad[0].error
    assert all(r.counts is not None for r in done if r.error is None)
