"""Continuous-batching server for GF(2)[x] products on one GPU.

Requests (operands a, b of any lengths) arrive one by one.  The server keeps a
FIFO of pending requests and a few CUDA streams.  Whenever a stream is free it
takes the pending requests that fit the device-memory budget (results plus
the batch workspace, see ``gf2x_batch_workspace_bytes``), launches them as one
``gf2x_mul_batch`` on that stream (one persistent kernel launch), and records
an event.  Requests that arrive while other batches run are admitted into the
next batch on another stream, so their work overlaps on the device; a batch
is complete when its event has fired.  Latency of a request = completion time
- arrival time, both on the host clock.

Admission: a request that could not run even alone within the budget (its
result, its staging buffers and a one-job batch workspace) is refused at
``submit`` with GF2X_ENOMEM and never queued.  A pending request can be
cancelled until a batch takes it.

Resident transforms: the forward transform of an operand b (Alg. 5's steps for
b, at the transform length of the product) can be kept on the device.  A
request names its b with ``b_key`` (any hashable value that stands for b's
contents; None: never reused).  The server counts how often the same
(b_key, nb) recurs at the same transform length; from the ``reuse_after``-th
time on it computes b's transform once (``gf2x_forward_transform``), keeps it
within a share of the budget (least recently used dropped), and runs the
requests with that b as ``gf2x_mul_transformed`` on the batch's stream,
skipping b's forward steps.  Other streams wait for the transform's event
before they use it.

Host operands: a request may carry page-locked host tensors instead of device
ones (``Request.host``).  The server then copies its operands to the device on
the batch's stream before the batch and the product back to a page-locked host
tensor after it, so a request's latency includes both transfers.

Outputs: a request without a caller-provided ``out`` gets one when a batch
takes it (device memory, or page-locked host memory for host requests), counted
against the budget while its batch runs; from then on it belongs to the caller.
So the memory a server holds is bounded by the batches in flight, however long
the queue.  ``on_done`` (optional) is called with every completed request, e.g.
to consume or drop its output.

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

from . import STATUS, Context, product_bits, transform_bits, workspace_bytes

GF2X_OK = 0
GF2X_ENOMEM = 3


@dataclass(eq=False)            # requests compare by identity (queue membership, cancel)
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
    host: bool = False          # a, b are page-locked host tensors; out is one too
    b_key: object = None        # identity of b's contents, for resident transforms (None: not reused)
    status: int = GF2X_OK       # GF2X_ENOMEM when refused at admission
    state: str = "new"          # new, pending, running, done, rejected, cancelled
    reused: bool = False        # ran with b's resident transform
    _dev_a: object = None
    _dev_b: object = None
    _dev_out: object = None


@dataclass
class _Batch:
    reqs: list
    stream: object
    event: object
    workspace: object
    bytes: int
    launched: float = field(default_factory=time.perf_counter)


def _words(bits: int) -> int:
    return (bits + 63) // 64


class Server:
    """Admit, batch and complete products; one batch in flight per stream."""

    def __init__(self, ctx: Context, streams: int = 3, memory_budget: int | None = None, max_batch: int = 512,
                 reserve_bytes: int = 2 << 30, reuse_after: int = 0, transform_share: float = 0.25, on_done=None):
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
        self.rejected: list = []
        self.cancelled: list = []
        self._next_batch = 0
        # resident transforms: key (b_key, nb, n) -> (transform, its event, its stream); recurrence counts
        self.reuse_after = reuse_after      # 0: never keep transforms
        self.transform_budget = int(self.budget * transform_share)
        self.transforms: collections.OrderedDict = collections.OrderedDict()
        self.transform_bytes = 0
        self.seen: collections.Counter = collections.Counter()
        self.on_done = on_done

    # ------------------------------------------------------------ requests
    def _request_bytes(self, r: Request) -> int:
        """Device bytes a request needs when it runs alone: its result, its
        staging buffers (host requests) and a one-job batch workspace."""
        nc = product_bits(r.na, r.nb)
        n = transform_bits(r.na, r.nb)
        staged = 8 * (_words(r.na) + _words(r.nb)) if r.host else 0
        return 8 * max(_words(nc), 1) + staged + (3 * ((n // 8 + 255) // 256 * 256) + 48 if n else 48) + 4096

    def submit(self, req: Request) -> int:
        """Queue a request; GF2X_OK, or GF2X_ENOMEM (refused, not queued) when it
        cannot run within the memory budget even alone."""
        import torch
        if not req.arrival:
            req.arrival = time.perf_counter()
        if self._request_bytes(req) > self.budget:
            req.status = GF2X_ENOMEM
            req.state = "rejected"
            req.done = time.perf_counter()
            self.rejected.append(req)
            return GF2X_ENOMEM
        nc = product_bits(req.na, req.nb)
        if req.out is not None and req.out.numel() < max(_words(nc), 1):
            req.out = None                          # too short: the server allocates one at launch
        req.state = "pending"
        self.pending.append(req)
        return GF2X_OK

    def cancel(self, req: Request) -> bool:
        """Withdraw a request that no batch has taken yet; False once it runs or ran."""
        if req.state != "pending":
            return False
        try:
            self.pending.remove(req)
        except ValueError:
            return False
        req.state = "cancelled"
        self.cancelled.append(req)
        return True

    @staticmethod
    def _cost1(r) -> int:
        """Workspace bytes one request adds to a batch (three n-bit buffers and its table row)."""
        n = transform_bits(r.na, r.nb)
        return 3 * ((n // 8 + 255) // 256 * 256) + 48 if n else 48

    # ------------------------------------------------------ resident transforms
    def _transform_key(self, r: Request):
        if r.host or r.b_key is None or not self.reuse_after or product_bits(r.na, r.nb) == 0:
            return None
        return (r.b_key, r.nb, transform_bits(r.na, r.nb))

    def _resident(self, r: Request, stream):
        """b's resident transform for this request (computing it on `stream` once
        b has recurred often enough), or None.  The caller runs on `stream`."""
        import torch
        key = self._transform_key(r)
        if key is None:
            return None
        if key in self.transforms:
            self.transforms.move_to_end(key)
            bhat, ev, owner = self.transforms[key]
            if owner is not stream:
                stream.wait_event(ev)                   # computed on another stream
                bhat.record_stream(stream)
            return bhat
        self.seen[key] += 1
        n = key[2]
        if self.seen[key] < self.reuse_after or n // 8 > self.transform_budget:
            return None
        while self.transforms and self.transform_bytes + n // 8 > self.transform_budget:
            _, (old, _, _) = self.transforms.popitem(last=False)     # least recently used
            self.transform_bytes -= old.numel() * 8
        bhat = torch.empty(n // 64, dtype=torch.int64, device=self.device)
        ws = torch.empty(self.ctx._lib.gf2x_transform_workspace_bytes(n), dtype=torch.uint8, device=self.device)
        self.ctx.forward_transform(r.b, r.nb, n, out=bhat, workspace=ws, stream=stream)
        ev = torch.cuda.Event()
        ev.record(stream)
        self.transforms[key] = (bhat, ev, stream)
        self.transform_bytes += n // 8
        return bhat

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
                    r.state = "done"
                    if r.host:                          # the device copies are no longer needed
                        r._dev_a = r._dev_b = r._dev_out = None
                    self.completed.append(r)
                    if self.on_done is not None:
                        self.on_done(r)
                finished += len(bt.reqs)
                self.in_use -= bt.bytes
                del self.inflight[k]
        for k, st in enumerate(self.streams):
            if k in self.inflight or not self.pending:
                continue
            take = []
            cost = 1024                                 # table alignment and reserved state
            while self.pending and len(take) < self.max_batch:
                r = self.pending[0]
                nw = max(_words(product_bits(r.na, r.nb)), 1)
                c = self._cost1(r) + (8 * (_words(r.na) + _words(r.nb) + nw) if r.host else 0)
                if r.out is None and not r.host:
                    c += 8 * nw                         # the output the server allocates at launch
                if take and self.in_use + cost + c > self.budget:
                    break
                take.append(self.pending.popleft())
                cost += c
            if not take:
                break
            with torch.cuda.stream(st):
                for r in take:                          # outputs, and host operands' copies on the batch's stream
                    if r.out is None:
                        nw = max(_words(product_bits(r.na, r.nb)), 1)
                        r.out = (torch.empty(nw, dtype=torch.int64, pin_memory=True) if r.host
                                 else torch.empty(nw, dtype=torch.int64, device=self.device))
                    if r.host:
                        r._dev_a = r.a.to(self.device, non_blocking=True)
                        r._dev_b = r.b.to(self.device, non_blocking=True)
                        r._dev_out = torch.empty(max(_words(product_bits(r.na, r.nb)), 1), dtype=torch.int64,
                                                 device=self.device)
                    else:
                        r._dev_a, r._dev_b, r._dev_out = r.a, r.b, r.out
                plain, reused = [], []
                for r in take:
                    bhat = self._resident(r, st)
                    (reused if bhat is not None else plain).append((r, bhat))
                jobs = [(r._dev_a, r.na, r._dev_b, r.nb, r._dev_out) for r, _ in plain]
                wsb = self.ctx.batch_workspace_bytes(jobs) if jobs else 256
                for r, _ in reused:
                    wsb = max(wsb, workspace_bytes(r.na, r.nb))
                cost = max(cost, wsb)
                if self.in_use + cost > self.budget and self.inflight:
                    for r in reversed(take):            # wait for memory to free up
                        self.pending.appendleft(r)
                    break
                ws = torch.empty(max(cost, 256), dtype=torch.uint8, device=self.device)
                if jobs:
                    self.ctx.mul_batch(jobs, workspace=ws, stream=st)
                for r, bhat in reused:                  # b's forward steps skipped
                    r.reused = True
                    self.ctx.mul_transformed(r._dev_a, r.na, bhat, r.nb, out=r._dev_out, workspace=ws, stream=st)
                for r in take:
                    if r.host:
                        r.out.copy_(r._dev_out, non_blocking=True)
                    r.state = "running"
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


__all__ = ["Server", "Request", "percentile", "GF2X_OK", "GF2X_ENOMEM", "STATUS"]
