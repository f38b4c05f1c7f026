"""Continuous-batching server for GF(2)[x] products on one GPU.

Requests (device-resident operands a, b of any lengths) arrive one by one.
The server keeps a FIFO of pending requests and a few CUDA streams.  Whenever
a stream is free it takes the pending requests that fit the device-memory
budget (results plus the batch workspace, see ``gf2x_batch_workspace_bytes``),
launches them as one ``gf2x_mul_batch`` on that stream, and records an event.
Requests that arrive while other batches run are admitted into the next batch
on another stream, so their work overlaps on the device; a batch is complete
when its event has fired.  Latency of a request = completion time - arrival
time, both on the host clock.

The library measures launch shapes the first time it meets a shape class,
which stalls that batch's stream; a server warms up on a representative mix
and then calls ``Context.tune_freeze()`` so that no request waits on a
measurement.

This module only schedules: every product runs in the library's kernels.
"""

from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

from . import Context, product_bits, transform_bits


@dataclass
class Request:
    a: object
    na: int
    b: object
    nb: int
    arrival: float = 0.0
    out: object = None
    done: float = 0.0
    batch_id: int = -1
    tag: object = None


@dataclass
class _Batch:
    reqs: list
    stream: object
    event: object
    workspace: object
    bytes: int
    launched: float = field(default_factory=time.perf_counter)


class Server:
    """Admit, batch and complete products; one batch in flight per stream."""

    def __init__(self, ctx: Context, streams: int = 3, memory_budget: int | None = None, max_batch: int = 512,
                 reserve_bytes: int = 2 << 30):
        import torch
        self.ctx = ctx
        self.device = torch.device("cuda", ctx.device)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(streams)]
        free, _ = torch.cuda.mem_get_info(self.device)
        self.budget = min(memory_budget or free, max(free - reserve_bytes, 1 << 28))
        self.max_batch = max_batch
        self.pending: collections.deque = collections.deque()
        self.inflight: dict = {}            # stream index -> _Batch
        self.in_use = 0
        self.completed: list = []
        self._next_batch = 0

    # ------------------------------------------------------------ requests
    def submit(self, req: Request):
        import torch
        if not req.arrival:
            req.arrival = time.perf_counter()
        nc = product_bits(req.na, req.nb)
        req.out = torch.empty(max((nc + 63) // 64, 1), dtype=torch.int64, device=self.device)
        self.pending.append(req)

    @staticmethod
    def _cost1(r) -> int:
        """Workspace bytes one request adds to a batch (three n-bit buffers and its table row)."""
        n = transform_bits(r.na, r.nb)
        return 3 * ((n // 8 + 255) // 256 * 256) + 48 if n else 48

    # ------------------------------------------------------------ progress
    def poll(self) -> int:
        """Retire finished batches and launch new ones; returns requests completed."""
        import torch
        finished = 0
        now = time.perf_counter()
        for k in list(self.inflight):
            bt = self.inflight[k]
            if bt.event.query():
                for r in bt.reqs:
                    r.done = now
                    self.completed.append(r)
                finished += len(bt.reqs)
                self.in_use -= bt.bytes
                del self.inflight[k]
        for k, st in enumerate(self.streams):
            if k in self.inflight or not self.pending:
                continue
            take = []
            cost = 1024                                 # table alignment and reserved state
            while self.pending and len(take) < self.max_batch:
                c = self._cost1(self.pending[0])
                if take and self.in_use + cost + c > self.budget:
                    break
                take.append(self.pending.popleft())
                cost += c
            if not take:
                break
            jobs = [(r.a, r.na, r.b, r.nb, r.out) for r in take]
            cost = max(cost, self.ctx.batch_workspace_bytes(jobs))
            if self.in_use + cost > self.budget and self.inflight:
                for r in reversed(take):             # wait for memory to free up
                    self.pending.appendleft(r)
                break
            ws = torch.empty(max(cost, 256), dtype=torch.uint8, device=self.device)
            with torch.cuda.stream(st):
                self.ctx.mul_batch(jobs, workspace=ws, stream=st)
                ev = torch.cuda.Event()
                ev.record(st)
            for r in take:
                r.batch_id = self._next_batch
            self._next_batch += 1
            self.inflight[k] = _Batch(take, st, ev, ws, cost)
            self.in_use += cost
        return finished

    def drain(self):
        while self.pending or self.inflight:
            self.poll()


def percentile(values, q):
    if not values:
        return None
    v = sorted(values)
    i = min(len(v) - 1, max(0, int(round(q / 100.0 * (len(v) - 1)))))
    return v[i]
