"""Host logic of the continuous-batching loop (paper_1409_0074_gb300/serve.py),
driven by a simulated device: admission by free slots and memory, FIFO
merging into batches, per-request routing of results, latency accounting."""
import numpy as np
import pytest

from paper_1409_0074_gb300.serve import (Request, Server, latency_summary, poisson_requests,
                                         run_stream)


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeDevice:
    """Slots and a memory budget (bytes per location); a batch finishes
    `cost_per_loc * M + fixed` seconds after submission.  Its 'prediction' of a
    location is a function of that location alone, so routing errors show."""

    def __init__(self, clock, slots=2, mem=10_000, bytes_per_loc=1, cost_per_loc=1e-3, fixed=1e-3):
        self.clock, self.slots, self.mem = clock, slots, mem
        self.bpl, self.cpl, self.fixed = bytes_per_loc, cost_per_loc, fixed
        self.inflight = {}
        self.max_inflight = 0
        self.next = 0
        self.submitted = []

    def submit(self, xref, n_loc):
        M = xref.shape[0]
        used = sum(v[2] for v in self.inflight.values())
        if len(self.inflight) >= self.slots or used + M * self.bpl > self.mem:
            return None
        h = self.next
        self.next += 1
        done = self.clock() + self.cpl * M + self.fixed
        mean = xref.sum(axis=1) * n_loc
        s2 = n_loc.astype(np.float64)
        self.inflight[h] = (done, (mean, s2), M * self.bpl)
        self.max_inflight = max(self.max_inflight, len(self.inflight))
        self.submitted.append(M)
        return h

    def poll(self, h):
        done, out, _ = self.inflight[h]
        if self.clock() < done:
            return None
        del self.inflight[h]
        return out


def _drive(server, clock, reqs, dt=1e-4, limit=100000):
    reqs = sorted(reqs, key=lambda r: r.arrival)
    i = 0
    for _ in range(limit):
        while i < len(reqs) and reqs[i].arrival <= clock.t:
            server.arrive(reqs[i])
            i += 1
        server.step()
        if i == len(reqs) and server.idle():
            return
        clock.t += dt
    raise AssertionError("the loop did not finish")


def _check_results(reqs):
    for r in reqs:
        assert r.done_at is not None
        np.testing.assert_array_equal(r.mean, r.xref.sum(axis=1) * r.n)
        np.testing.assert_array_equal(r.s2, np.full(r.xref.shape[0], float(r.n)))


def test_every_request_gets_its_own_results():
    rng = np.random.default_rng(0)
    clock = FakeClock()
    dev = FakeDevice(clock, slots=3, mem=5000)
    srv = Server(dev, max_batch=1024, clock=clock)
    reqs = poisson_requests(rng, rate=2000.0, count=300, p=3, sizes=(1, 700))
    _drive(srv, clock, reqs)
    assert len(srv.done) == len(reqs)
    _check_results(reqs)
    assert max(dev.submitted) <= 1024


def test_admission_respects_slots_and_memory():
    rng = np.random.default_rng(1)
    clock = FakeClock()
    dev = FakeDevice(clock, slots=2, mem=800, cost_per_loc=2e-3)
    srv = Server(dev, max_batch=800, clock=clock)
    reqs = poisson_requests(rng, rate=5000.0, count=100, p=2, sizes=(50, 400))
    _drive(srv, clock, reqs, dt=1e-3)
    assert dev.max_inflight <= 2
    assert len(srv.done) == 100
    _check_results(reqs)


def test_requests_are_merged_in_arrival_order():
    clock = FakeClock()
    dev = FakeDevice(clock, slots=1, mem=10_000, cost_per_loc=0.0, fixed=1.0)
    srv = Server(dev, max_batch=100, clock=clock)
    reqs = [Request(k, np.full((30, 2), float(k)), 50, 0.0) for k in range(5)]
    for r in reqs:
        srv.arrive(r)
    srv.step()
    # one slot: the first batch takes the first three requests (90 locations)
    assert dev.submitted == [90]
    assert [r.rid for r in srv.inflight[0].requests] == [0, 1, 2]
    clock.t = 1.5
    srv.step()
    assert dev.submitted == [90, 60]
    clock.t = 3.0
    srv.step()
    assert srv.idle()
    _check_results(reqs)


def test_late_arrival_joins_while_others_run():
    """Continuous batching: a request that arrives while a long batch is on the
    device is admitted into a free slot at once, not after that batch."""
    clock = FakeClock()
    dev = FakeDevice(clock, slots=2, mem=10_000, cost_per_loc=1e-2, fixed=0.0)
    srv = Server(dev, max_batch=4096, clock=clock)
    big = Request(0, np.ones((1000, 2)), 50, 0.0)      # 10 s on the device
    small = Request(1, np.ones((10, 2)), 50, 0.5)      # arrives at 0.5 s, 0.1 s of work
    _drive(srv, clock, [big, small], dt=1e-2)
    assert small.done_at < big.done_at
    assert small.latency == pytest.approx(0.1, abs=0.02)
    _check_results([big, small])


def test_oversized_batch_waits_for_memory():
    clock = FakeClock()
    dev = FakeDevice(clock, slots=4, mem=1000, cost_per_loc=1e-3, fixed=0.0)
    srv = Server(dev, max_batch=1000, clock=clock)
    a = Request(0, np.ones((700, 2)), 30, 0.0)
    b = Request(1, np.ones((600, 2)), 30, 0.0)
    srv.arrive(a)
    srv.arrive(b)
    srv.step()
    assert dev.submitted == [700]        # b does not fit beside a
    _drive(srv, clock, [], dt=1e-3)
    assert dev.submitted == [700, 600]
    assert b.done_at >= a.done_at
    _check_results([a, b])


def test_latency_summary():
    reqs = [Request(k, np.zeros((10, 2)), 30, 0.0) for k in range(100)]
    for k, r in enumerate(reqs):
        r.done_at = (k + 1) * 1e-3
    s = latency_summary(reqs, wall=0.1)
    assert s["requests"] == 100 and s["locations"] == 1000
    assert s["p50_ms"] == pytest.approx(50.5)
    assert s["p99_ms"] == pytest.approx(99.01)
    assert s["locations_per_s"] == pytest.approx(10000.0)


def test_run_stream_real_clock():
    import time
    rng = np.random.default_rng(2)
    dev = FakeDevice(time.perf_counter, slots=2, mem=100_000, cost_per_loc=1e-6, fixed=1e-4)
    srv = Server(dev, max_batch=4096)
    reqs = poisson_requests(rng, rate=5000.0, count=50, p=2, sizes=(1, 64))
    wall = run_stream(srv, reqs)
    assert wall > 0 and len(srv.done) == 50
    _check_results(reqs)
