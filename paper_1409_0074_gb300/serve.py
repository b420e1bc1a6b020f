"""Continuous-batching request loop over a serving context (laGP_ctx_*).

Requests (a batch of predictive locations each, with its own local design
size n) arrive over time.  The loop keeps a FIFO queue of arrived requests and
a set of in-flight device batches.  Whenever the context has a free slot and a
free arena region, the requests at the head of the queue are merged into one
device batch (their locations concatenated, each location carrying its
request's n), up to `max_batch` locations, and submitted; batches run
concurrently on the device, one stream per slot.  A request that arrives while
others are on the GPU joins the next batch that is admitted.  Completed batches
are split back into their requests and each request's latency (arrival to
results in host memory) is recorded.

The loop logic is independent of the device: `CtxBackend` drives the CUDA
library, and any object with the same submit / poll interface (a simulated
device in the CPU tests) can stand in for it.
"""
import time
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class Request:
    rid: int
    xref: np.ndarray            # [M][p] float64
    n: int                      # local design size of every location of the request
    arrival: float              # seconds, on the loop's clock
    mean: Optional[np.ndarray] = None
    s2: Optional[np.ndarray] = None
    done_at: Optional[float] = None

    @property
    def latency(self):
        return None if self.done_at is None else self.done_at - self.arrival


@dataclass
class Batch:
    requests: List[Request]
    offsets: List[int]
    handle: object
    submitted: float
    locations: int


class CtxBackend:
    """Submits merged batches to a lagp.Context; reuses one set of page-locked
    host buffers per in-flight slot."""

    def __init__(self, ctx, max_batch, slots):
        import torch
        self.ctx, self.max_batch, self.p = ctx, max_batch, ctx.p

        def pinned(shape, dtype):
            return torch.empty(shape, dtype=dtype).pin_memory().numpy()

        self.free = [dict(xref=pinned((max_batch, self.p), torch.float64),
                          nloc=pinned((max_batch,), torch.int32),
                          mean=pinned((max_batch,), torch.float64),
                          s2=pinned((max_batch,), torch.float64)) for _ in range(slots)]

    def submit(self, xref, n_loc):
        """Returns a handle, or None when no slot / buffer / arena region is free."""
        if not self.free:
            return None
        M = xref.shape[0]
        if M > self.max_batch:
            raise ValueError("batch larger than max_batch")
        buf = self.free.pop()
        bx = buf["xref"][:M]
        bx[...] = xref
        bn = buf["nloc"][:M]
        bn[...] = n_loc
        n = int(n_loc.max())
        uniform = bool((n_loc == n).all())
        t = self.ctx.submit(bx, n, buf["mean"][:M], buf["s2"][:M],
                            n_loc=None if uniform else bn)
        if t is None:
            self.free.append(buf)
            return None
        return (t, buf, M)

    def poll(self, handle):
        """(mean, s2) copies once done, else None."""
        t, buf, M = handle
        if not self.ctx.poll(t):
            return None
        out = (buf["mean"][:M].copy(), buf["s2"][:M].copy())
        self.free.append(buf)
        return out


class Server:
    def __init__(self, backend, max_batch=4096, clock=time.perf_counter):
        self.backend, self.max_batch, self.clock = backend, max_batch, clock
        self.queue: List[Request] = []
        self.inflight: List[Batch] = []
        self.done: List[Request] = []
        self.batches = 0
        self.batch_sizes: List[int] = []

    def arrive(self, req: Request):
        if req.xref.shape[0] > self.max_batch:
            raise ValueError("request of %d locations exceeds max_batch %d"
                             % (req.xref.shape[0], self.max_batch))
        self.queue.append(req)

    def _collect(self):
        still = []
        for b in self.inflight:
            r = self.backend.poll(b.handle)
            if r is None:
                still.append(b)
                continue
            mean, s2 = r
            now = self.clock()
            for req, o in zip(b.requests, b.offsets):
                m = req.xref.shape[0]
                req.mean, req.s2, req.done_at = mean[o:o + m], s2[o:o + m], now
                self.done.append(req)
        self.inflight = still

    def _admit(self):
        while self.queue:
            take, total = [], 0
            for req in self.queue:
                m = req.xref.shape[0]
                if take and total + m > self.max_batch:
                    break
                take.append(req)
                total += m
            xref = np.concatenate([r.xref for r in take], axis=0)
            n_loc = np.concatenate([np.full(r.xref.shape[0], r.n, np.int32) for r in take])
            h = self.backend.submit(xref, n_loc)
            if h is None:
                return          # no slot or memory: wait for a batch to finish
            offs = np.cumsum([0] + [r.xref.shape[0] for r in take[:-1]]).tolist()
            self.inflight.append(Batch(take, offs, h, self.clock(), total))
            self.batches += 1
            self.batch_sizes.append(total)
            del self.queue[:len(take)]

    def step(self):
        """One pass: collect finished batches, then admit queued requests."""
        self._collect()
        self._admit()

    def idle(self):
        return not self.queue and not self.inflight


def run_stream(server: Server, requests: List[Request], poll_sleep=0.0002):
    """Feeds `requests` (sorted by arrival, times relative to the start) to the
    server in real time and runs it until every request is done.  Returns the
    wall time from the first arrival to the last completion."""
    reqs = sorted(requests, key=lambda r: r.arrival)
    t0 = server.clock()
    for r in reqs:
        r.arrival += t0
    i = 0
    while i < len(reqs) or not server.idle():
        now = server.clock()
        while i < len(reqs) and reqs[i].arrival <= now:
            server.arrive(reqs[i])
            i += 1
        server.step()
        if server.inflight or i < len(reqs):
            time.sleep(poll_sleep)
    return server.clock() - t0


def poisson_requests(rng, rate, count, p, sizes=(1, 4096), ns=(30, 50, 100), t_start=0.0):
    """`count` requests with exponential inter-arrival times (mean 1/rate s),
    sizes log-uniform in [sizes[0], sizes[1]] locations, n uniform over `ns`,
    locations iid uniform on [0, 1]^p."""
    out, t = [], t_start
    lo, hi = np.log(sizes[0]), np.log(sizes[1] + 1)
    for k in range(count):
        t += rng.exponential(1.0 / rate)
        m = int(np.exp(rng.uniform(lo, hi)))
        m = max(sizes[0], min(sizes[1], m))
        out.append(Request(k, rng.random((m, p)), int(rng.choice(ns)), t))
    return out


def latency_summary(reqs: List[Request], wall):
    lat = np.array([r.latency for r in reqs]) * 1e3
    locs = sum(r.xref.shape[0] for r in reqs)
    return {"requests": len(reqs), "locations": locs, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
            "locations_per_s": locs / wall, "wall_s": wall}
