"""Serving loop: sort requests of mixed sizes as they arrive, with continuous
batching on the GPU.

Requests are admitted against a device-memory budget into a resident arena.
A scheduler thread groups the admitted requests of one kind (keys only, or keys
with payloads) into a batch whenever one of the CUDA streams has room, lays the
batch out contiguously in the arena, lets each request write its data into its
slot (the request's fill callback), and sorts the whole batch with one
isort_segmented call -- every request is one range, so each result is exactly
what a sort of that request alone gives. A batch of one request (a stream was
free when it arrived and nothing else was waiting) runs the plain sort
instead, which has less fixed cost per launch. Batches on different streams overlap
on the device; requests that arrive while others are on the GPU join the next
batch as soon as a stream and arena space are free. One completion thread per
stream waits for its batches in order, stamps each request's completion time,
runs its done callback and frees its arena space.

Latency is completion time minus arrival time (host perf_counter clock).
The same loop with batching switched off (max_batch_requests=1, one stream)
is the sequential baseline: one plain sort per request, in arrival order.
"""
from __future__ import annotations

import bisect
import collections
import threading
import time
from dataclasses import dataclass, field
from typing import Callable, Optional

from . import _lib, load, set_workspace, sort_keys, sort_pairs, sort_segmented, stream_status
from . import segmented_workspace_size, workspace_size


@dataclass
class Request:
    rid: int
    n: int                      # keys
    payload: bool               # uint32 payloads travel with the keys
    arrival: float              # perf_counter seconds
    fill: Callable              # fill(keys_view, vals_view_or_None, cuda_stream)
    done: Optional[Callable] = None  # done(request, keys_view, vals_view) on completion
    start: float = 0.0          # batch launch time
    finish: float = 0.0         # completion time
    batch: int = -1
    keys: object = None         # arena views while in flight
    vals: object = None
    _alloc: list = field(default_factory=list)


class Arena:
    """First-fit allocator over one device buffer (host-side bookkeeping only)."""

    ALIGN = 256

    def __init__(self, nbytes: int, device: str = "cuda"):
        import torch
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.size = nbytes
        self.free = [(0, nbytes)]  # sorted (offset, size)
        self.used = 0

    def alloc(self, nbytes: int):
        need = (nbytes + self.ALIGN - 1) // self.ALIGN * self.ALIGN
        for i, (off, sz) in enumerate(self.free):
            if sz >= need:
                if sz == need:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + need, sz - need)
                self.used += need
                return off, need
        return None

    def release(self, off: int, size: int):
        i = bisect.bisect_left(self.free, (off, 0))
        self.free.insert(i, (off, size))
        self.used -= size
        # coalesce with neighbours
        if i + 1 < len(self.free) and self.free[i][0] + self.free[i][1] == self.free[i + 1][0]:
            self.free[i] = (self.free[i][0], self.free[i][1] + self.free[i + 1][1])
            self.free.pop(i + 1)
        if i > 0 and self.free[i - 1][0] + self.free[i - 1][1] == self.free[i][0]:
            self.free[i - 1] = (self.free[i - 1][0], self.free[i - 1][1] + self.free[i][1])
            self.free.pop(i)

    def view(self, off: int, nbytes: int, dtype):
        return self.buf[off:off + nbytes].view(dtype)


class SortServer:
    def __init__(self, budget_bytes: int, num_streams: int = 4, max_batch_keys: int = 1 << 26,
                 max_batch_requests: int = 4096, batching: bool = True):
        import torch
        load()
        self.torch = torch
        self.batching = batching
        self.max_batch_keys = max_batch_keys
        self.max_batch_requests = max_batch_requests if batching else 1
        self.num_streams = num_streams if batching else 1
        self.streams = [torch.cuda.Stream() for _ in range(self.num_streams)]
        # per-stream workspace, bound once (no allocation while serving)
        # (a batch of one request runs the plain sort, so both kinds must fit)
        ws = max(workspace_size(max_batch_keys, 32, 32, 8), workspace_size(max_batch_keys, 32, 0, 8))
        if batching:
            ws = max(ws, segmented_workspace_size(max_batch_requests, max_batch_keys, 32, 32),
                     segmented_workspace_size(max_batch_requests, max_batch_keys, 32, 0))
        self.ws = [torch.empty(ws, dtype=torch.uint8, device="cuda") for _ in self.streams]
        for s, w in zip(self.streams, self.ws):
            set_workspace(w, stream=s)
        self.arena = Arena(budget_bytes)
        self.queue = collections.deque()
        self.cv = threading.Condition()
        self.inflight = [collections.deque() for _ in self.streams]  # (event, requests, allocs)
        self.stream_cv = [threading.Condition() for _ in self.streams]
        self.stop = False
        self.batches = 0
        self.errors = []
        self.completed = []
        self.failed = 0
        self.submitted = 0
        self.rejected = []
        self.cancelled = []
        self.sched = threading.Thread(target=self._schedule, daemon=True)
        self.waiters = [threading.Thread(target=self._complete, args=(i,), daemon=True)
                        for i in range(self.num_streams)]
        self.sched.start()
        for w in self.waiters:
            w.start()

    # ---- client side
    def submit(self, req: Request):
        nbytes = req.n * (8 if req.payload else 4)
        if req.n > self.max_batch_keys or nbytes > self.arena.size:
            self.rejected.append(req)  # can never fit: refused at admission
            return False
        with self.cv:
            self.submitted += 1
            self.queue.append(req)
            self.cv.notify()
        return True

    def cancel(self, req: Request) -> bool:
        """Withdraw a request that is still waiting in the queue. Returns True if
        it was withdrawn (it will never run and its done callback is never
        called); a request already in a batch runs to completion (False)."""
        with self.cv:
            for i, r in enumerate(self.queue):
                if r is req:
                    del self.queue[i]
                    self.submitted -= 1  # close() waits for what is still admitted
                    self.cancelled.append(req)
                    self.cv.notify_all()
                    return True
        return False

    def close(self, wait: bool = True):
        if wait:  # until every admitted request has completed (or failed to launch)
            with self.cv:
                while len(self.completed) + self.failed < self.submitted and not self.errors:
                    self.cv.wait(0.01)
        self.stop = True
        with self.cv:
            self.cv.notify_all()
        for c in self.stream_cv:
            with c:
                c.notify_all()
        self.sched.join()
        for w in self.waiters:
            w.join()
        for s in self.streams:
            set_workspace(None, stream=s)

    # ---- scheduler
    def _free_stream(self):
        best, best_len = None, None
        for i in range(self.num_streams):
            ln = len(self.inflight[i])
            if ln < 2 and (best is None or ln < best_len):  # at most 2 batches queued per stream
                best, best_len = i, ln
        return best

    def _schedule(self):
        while not self.stop:
            with self.cv:
                while not self.queue and not self.stop:
                    self.cv.wait(0.005)
                if self.stop:
                    return
                si = self._free_stream()
                if si is None:
                    self.cv.wait(0.0002)
                    continue
                # candidates: the oldest request's kind, in arrival order
                kind = self.queue[0].payload
                batch, keys_total = [], 0
                for r in self.queue:
                    if len(batch) >= self.max_batch_requests:
                        break
                    if r.payload != kind:
                        if not self.batching:
                            break
                        continue
                    if batch and keys_total + r.n > self.max_batch_keys:
                        break
                    batch.append(r)
                    keys_total += r.n
                # admission against the budget: one contiguous region per batch
                # (keys, and payloads); shrink the batch until it fits
                while batch:
                    a = self.arena.alloc(keys_total * 4)
                    b = self.arena.alloc(keys_total * 4) if kind else (0, 0)
                    if a is not None and b is not None:
                        break
                    if a is not None:
                        self.arena.release(*a)
                    if b is not None and kind:
                        self.arena.release(*b)
                    keys_total -= batch.pop().n
                if not batch:
                    self.cv.wait(0.0005)  # out of budget: wait for completions
                    continue
                taken = set(id(r) for r in batch)
                self.queue = collections.deque(r for r in self.queue if id(r) not in taken)
                batch[0]._alloc = [a] + ([b] if kind else [])
            try:
                self._launch(si, batch, kind, keys_total)
            except Exception as e:  # surfaced through .errors
                self.errors.append(e)
                with self.cv:
                    for off, sz in batch[0]._alloc:
                        self.arena.release(off, sz)
                    self.failed += len(batch)
                    self.cv.notify_all()

    def _launch(self, si, batch, kind, keys_total):
        torch = self.torch
        stream = self.streams[si]
        self.batches += 1
        bid = self.batches
        now = time.perf_counter()
        (ka, _), vreg = batch[0]._alloc[0], (batch[0]._alloc[1] if kind else None)
        keys = self.arena.view(ka, keys_total * 4, torch.uint32)
        vals = self.arena.view(vreg[0], keys_total * 4, torch.uint32) if kind else None
        with torch.cuda.stream(stream):
            offs, o = [0], 0
            for r in batch:  # each request's data goes straight into its slot
                r.start, r.batch = now, bid
                r.keys = keys[o:o + r.n]
                r.vals = vals[o:o + r.n] if kind else None
                r.fill(r.keys, r.vals, stream)
                o += r.n
                offs.append(o)
            if self.batching and len(batch) > 1:
                d_off = torch.tensor(offs, dtype=torch.int64).to("cuda", non_blocking=True)
                sort_segmented(keys, d_off, vals)
            else:
                # a lone request (the common case at light load) or the sequential
                # baseline: the plain sort, without the segmented sort's fixed
                # cost (range classes, offsets upload)
                for r in batch:
                    if kind:
                        sort_pairs(r.keys, r.vals, 8)
                    else:
                        sort_keys(r.keys, 8)
            ev = torch.cuda.Event()
            ev.record(stream)
        with self.stream_cv[si]:
            self.inflight[si].append((ev, batch, batch[0]._alloc))
            self.stream_cv[si].notify()

    # ---- completion
    def _complete(self, si):
        while True:
            with self.stream_cv[si]:
                while not self.inflight[si] and not self.stop:
                    self.stream_cv[si].wait(0.005)
                if not self.inflight[si]:
                    return
                ev, batch, extra = self.inflight[si][0]
            ev.synchronize()
            t = time.perf_counter()
            st = stream_status(self.streams[si])
            if st != _lib.OK:
                self.errors.append(RuntimeError(f"stream {si}: {_lib.STATUS.get(st, st)}"))
            for r in batch:
                r.finish = t
                if r.done:
                    r.done(r, r.keys, r.vals)
            with self.cv:
                for r in batch:
                    r.keys = r.vals = None
                for off, sz in extra:  # the batch's regions
                    self.arena.release(off, sz)
                self.completed.extend(batch)
                self.cv.notify_all()
            with self.stream_cv[si]:
                self.inflight[si].popleft()
                self.stream_cv[si].notify_all()


def latency_summary(reqs):
    import numpy as np
    lat = np.array([r.finish - r.arrival for r in reqs]) * 1e3
    keys = sum(r.n for r in reqs)
    span = max(r.finish for r in reqs) - min(r.arrival for r in reqs) if reqs else 0.0
    return {"requests": len(reqs), "keys": int(keys),
            "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
            "mean_ms": float(lat.mean()) if len(lat) else None,
            "keys_per_s": keys / span if span > 0 else None}


def drive(server: SortServer, arrivals, sizes, payload, make_fill, duration_s: float,
          done=None):
    """Release requests at their arrival times (relative seconds) for duration_s;
    returns the list of submitted requests."""
    t0 = time.perf_counter()
    reqs = []
    for rid, (at, n, pay) in enumerate(zip(arrivals, sizes, payload)):
        if at > duration_s:
            break
        now = time.perf_counter() - t0
        if at > now:
            time.sleep(at - now)
        r = Request(rid=rid, n=int(n), payload=bool(pay), arrival=time.perf_counter(),
                    fill=make_fill(rid, int(n), bool(pay)), done=done)
        if server.submit(r):
            reqs.append(r)
    return reqs
