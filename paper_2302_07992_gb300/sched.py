"""Request scheduler of the serving loop: admission, batching, completion, cancellation,
failure handling and request metrics, independent of the device.

The scheduler decides WHICH requests run together and WHEN; an executor runs a batch.
``serve.CudaExecutor`` launches a batch as one plan per operation on its own CUDA
stream; tests drive the same scheduler with a host-thread executor whose delays and
failures they inject.  The executor interface:

  slots                  batches that may be in flight at once
  launch(reqs) -> h      start a batch of same-kind requests (may raise)
  ready(h) -> bool       the batch has finished (non-blocking)
  wait(h)                block until the batch has finished
  results(h) -> [dict]   per request: its outputs plus "info" (b, capacity, embedded,
                         extracted, hist, status); may raise when the batch failed
  discard(result)        give back the buffers of a result nobody will read
  release(h)             the batch's resources may be reused

Request statuses: "ok"; "capacity" (encode: the message was longer than the capacity
and only the capacity was embedded); "cancelled" (cancel() before completion: a
queued request never runs, an in-flight one runs and its result is discarded);
"rejected" (the queue was full on arrival); "error" (the launch or the batch failed;
the error text is in Request.error).  Every request ends in exactly one of them.
"""
from __future__ import annotations

import functools
import gc
import json
import math
import time
from collections import Counter, deque
from dataclasses import dataclass, field
from typing import Any, Callable

import numpy as np

STATUSES = ("ok", "capacity", "cancelled", "rejected", "error")


@dataclass
class Request:
    rid: int
    kind: str                      # "encode" or "decode"
    params: Any                    # rdhei.Params
    image: Any                     # host uint8 H x W (original or marked), pinned for the GPU executor
    payload: Any = None            # encode: packed message
    nbits: int = 0                 # encode: message bits; decode: bits to extract
    b: int = 0                     # decode: the public b
    lmr_map: Any = None            # LMR decode: packed rotated map
    lmr_eta: Any = None
    state: int = 0                 # decode: handle of device-resident maps kept by an earlier encode
    keep_state: bool = False       # encode: keep the LMR maps on the device, return a handle
    arrival: float = 0.0           # seconds on the scheduler clock
    done: float = -1.0
    status: str = ""
    error: str = ""
    result: dict = field(default_factory=dict)

    @functools.cached_property
    def pixels(self) -> int:
        H, W = self.image.shape
        return int(H) * int(W)

    @functools.cached_property
    def _bytes(self) -> int:
        N = self.pixels
        words = ((N + 31) // 32) * 4
        msg = ((self.nbits + 31) // 32) * 4 + 4
        return 4 * N + 2 * words + 2 * msg + N + N // 4 + 4096

    def device_bytes(self) -> int:
        """Device memory the request holds while in flight (buffers + workspace share)."""
        return self._bytes


class _InFlight:
    def __init__(self, handle, reqs, t_launch, seq):
        self.handle, self.reqs, self.t_launch, self.seq = handle, reqs, t_launch, seq


# latency histogram buckets: 0.05 ms * 2^k, k = 0 .. 19 (about 26 s), plus overflow
LAT_EDGES_MS = [0.05 * 2.0 ** k for k in range(20)]


class Scheduler:
    def __init__(self, executor, budget_bytes: float = 40e9, max_batch: int = 64,
                 max_batch_pixels: int = 1 << 27, max_queue: int | None = None,
                 clock: Callable[[], float] = time.perf_counter, admit_window_ms: float = 0.0):
        self.ex = executor
        self.budget = float(budget_bytes)
        # while a batch is on the device, hold new requests for up to this long so that
        # they leave together (an idle device takes the first request at once)
        self.admit_window = admit_window_ms * 1e-3
        self.max_batch = max_batch
        self.max_batch_pixels = max_batch_pixels
        self.max_queue = max_queue
        self.clock = clock
        self.in_use = 0.0
        self.inflight: list[_InFlight] = []
        self.queue: deque[Request] = deque()
        self.completed: list[Request] = []
        self.batches: list[dict] = []           # one record per launched batch
        self.cancelled: set[int] = set()
        self.consume = None
        self.t0 = None
        self._seq = 0

    def now(self) -> float:
        return self.clock() - self.t0

    def cancel(self, rid: int):
        """Cancel request rid: dropped if still queued, result discarded if in flight."""
        self.cancelled.add(rid)

    # ------------------------------------------------------------- completion --
    def _finish(self, r: Request, status: str, t: float, error: str = ""):
        r.status, r.done, r.error = status, t, error
        self.completed.append(r)
        if self.consume is not None and status in ("ok", "capacity"):
            self.consume(r)

    def _retire_one(self, f: _InFlight):
        t = self.now()
        rec = {"batch": f.seq, "kind": f.reqs[0].kind, "requests": len(f.reqs),
               "pixels": sum(r.pixels for r in f.reqs), "launch_ms": f.t_launch * 1e3, "done_ms": t * 1e3}
        try:
            outs = self.ex.results(f.handle)
            err = ""
        except Exception as e:                  # the batch failed on the device or in a copy
            outs, err = None, f"{type(e).__name__}: {e}"
        for r in f.reqs:
            self.in_use -= r.device_bytes()
        if outs is None:
            for r in f.reqs:
                self._finish(r, "error", t, err)
        else:
            for r, o in zip(f.reqs, outs):
                if r.rid in self.cancelled:
                    self.ex.discard(o)
                    r.result = {"info": o.get("info")}
                    self._finish(r, "cancelled", t)
                    continue
                r.result = o
                st = (o.get("info") or {}).get("status", 0)
                self._finish(r, "capacity" if st == 2 else "ok", t)
            infos = [o.get("info") or {} for o in outs]
            rec["b_hist"] = dict(sorted(Counter(int(i.get("b", 0)) for i in infos).items()))
            if f.reqs[0].kind == "encode":
                rec["embedded_bits"] = int(sum(int(i.get("embedded", 0)) for i in infos))
                rec["der_bpp"] = rec["embedded_bits"] / max(1, rec["pixels"])
        rec["status"] = dict(Counter(r.status for r in f.reqs))
        if err:
            rec["error"] = err
        self.batches.append(rec)
        self.ex.release(f.handle)

    def _retire(self, block: bool = False):
        still = []
        for f in self.inflight:
            if block or self.ex.ready(f.handle):
                self.ex.wait(f.handle)
                self._retire_one(f)
                block = False
            else:
                still.append(f)
        self.inflight = still

    # -------------------------------------------------------------- admission --
    def _enqueue(self, r: Request):
        if r.rid in self.cancelled:
            self._finish(r, "cancelled", self.now())
        elif self.max_queue is not None and len(self.queue) >= self.max_queue:
            self._finish(r, "rejected", self.now(), "queue full")
        else:
            self.queue.append(r)

    def _admit_batch(self) -> list[Request]:
        """Up to max_batch same-kind requests from the head of the queue that fit the
        memory budget (a request larger than the whole budget runs alone)."""
        while self.queue and self.queue[0].rid in self.cancelled:
            self._finish(self.queue.popleft(), "cancelled", self.now())
        if not self.queue or len(self.inflight) >= self.ex.slots:
            return []
        if (self.admit_window > 0 and self.inflight and self.now() - self.queue[0].arrival < self.admit_window
                and len(self.queue) < self.max_batch):
            return []
        kind = self.queue[0].kind
        batch, px = [], 0
        while self.queue and len(batch) < self.max_batch:
            r = self.queue[0]
            if r.rid in self.cancelled:
                self._finish(self.queue.popleft(), "cancelled", self.now())
                continue
            if r.kind != kind or px + r.pixels > self.max_batch_pixels and batch:
                break
            need = r.device_bytes()
            held = getattr(self.ex, "state_bytes", lambda: 0)()   # device-resident state of earlier requests
            if self.in_use + held + need > self.budget and (batch or self.inflight):
                break
            self.queue.popleft()
            self.in_use += need
            batch.append(r)
            px += r.pixels
        return batch

    def _launch(self, batch: list[Request]):
        t = self.now()
        try:
            h = self.ex.launch(batch)
        except Exception as e:
            for r in batch:
                self.in_use -= r.device_bytes()
            err = f"{type(e).__name__}: {e}"
            for r in batch:
                self._finish(r, "error", t, err)
            self.batches.append({"batch": self._seq, "kind": batch[0].kind, "requests": len(batch),
                                 "pixels": sum(r.pixels for r in batch), "launch_ms": t * 1e3, "done_ms": t * 1e3,
                                 "status": {"error": len(batch)}, "error": err})
            self._seq += 1
            return
        self.inflight.append(_InFlight(h, batch, t, self._seq))
        self._seq += 1

    # ------------------------------------------------------------------- loop --
    def run(self, requests: list[Request], realtime: bool = True, consume=None) -> list[Request]:
        """Serve requests whose `arrival` is on the scheduler clock (seconds from
        start).  realtime=False admits everything at once (arrival times ignored).
        consume(r), if given, is called as each request completes successfully.
        Returns every request, each with its final status, in completion order."""
        self.consume = consume
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        self.t0 = self.clock()
        if not realtime:
            for r in pending:
                r.arrival = 0.0
        # no cyclic garbage collection inside the loop: a full collection over the
        # requests' objects pauses the loop for milliseconds (a latency tail)
        gc_was_enabled = gc.isenabled()
        gc.disable()
        try:
            self._loop(pending)
        finally:
            if gc_was_enabled:
                gc.enable()
        return self.completed

    def _loop(self, pending: deque):
        while pending or self.queue or self.inflight:
            now = self.now()
            while pending and pending[0].arrival <= now:
                self._enqueue(pending.popleft())
            self._retire()
            launched = False
            while True:
                b = self._admit_batch()
                if not b:
                    break
                self._launch(b)
                launched = True
            if launched:
                continue
            if self.inflight and (len(self.inflight) >= self.ex.slots or not (pending or self.queue)):
                self._retire(block=True)          # slots busy or nothing else to do: wait for the oldest
            elif pending and not self.queue:
                # idle until the next arrival (or a completion)
                time.sleep(max(0.0, min(pending[0].arrival - self.now(), 2e-4)))
            elif self.queue and self.inflight:
                time.sleep(2e-5)                  # the budget is held by running batches, or the window is open

    # ---------------------------------------------------------------- metrics --
    def metrics(self) -> dict:
        """Request counts by status, latency of the served requests (p50 / p99 / mean and
        a histogram over LAT_EDGES_MS), sustained Mpx/s and the number of batches."""
        served = [r for r in self.completed if r.status in ("ok", "capacity")]
        out = {"requests": len(self.completed), "status": {s: sum(r.status == s for r in self.completed)
                                                           for s in STATUSES},
               "batches": len(self.batches)}
        out.update(latency_stats(served) if served else {"p50_ms": None, "p99_ms": None, "mean_ms": None,
                                                         "sustained_mpx": None})
        lat = [(r.done - r.arrival) * 1e3 for r in served]
        counts = [0] * (len(LAT_EDGES_MS) + 1)
        for v in lat:
            k = 0 if v <= LAT_EDGES_MS[0] else min(len(LAT_EDGES_MS), int(math.ceil(math.log2(v / LAT_EDGES_MS[0]))))
            counts[k] += 1
        out["latency_hist"] = {"upper_edges_ms": LAT_EDGES_MS, "counts": counts}
        return out

    def jsonl(self) -> str:
        """The batch records and a final metrics record, one JSON object per line."""
        lines = [json.dumps({"type": "batch", **b}) for b in self.batches]
        lines.append(json.dumps({"type": "metrics", **self.metrics()}))
        return "\n".join(lines) + "\n"


def latency_stats(done: list[Request]) -> dict:
    """p50 / p99 / mean latency (arrival -> completion) and sustained Mpx/s of the
    requests that were served (cancelled, rejected and failed requests excluded)."""
    done = [r for r in done if r.status in ("", "ok", "capacity")]
    lat = np.array([r.done - r.arrival for r in done]) * 1e3
    px = sum(r.pixels for r in done)
    span = max(r.done for r in done) - min(r.arrival for r in done)
    return {"requests": len(done), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "sustained_mpx": px / span / 1e6 if span > 0 else None}
