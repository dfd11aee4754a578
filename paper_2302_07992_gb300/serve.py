"""Continuous-batching request loop for encode and decode requests.

  encode request: an original image and a message -> rdhei_label_encrypt + rdhei_embed
                  -> marked image (and, for LMR, the rotated maps);
  decode request: a marked image (+ LMR maps) -> rdhei_extract + rdhei_decrypt_recover
                  -> message bits and recovered image.

Requests are admitted in arrival order while the device-memory budget and the number
of in-flight batches allow.  Each admitted group of same-kind requests becomes one
batch: one plan per operation over all its images, launched on its own stream, with
host<->device copies on that stream.  New batches are formed and launched while
earlier ones run, so work of requests that arrive while others are on the GPU
overlaps on the device.  A request's latency is arrival -> its batch's completion
(results back in host memory).  All work is in the library's kernels; this module
marshals buffers, plans and streams.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import rdhei as rd


@dataclass
class Request:
    rid: int
    kind: str                      # "encode" or "decode"
    params: rd.Params
    image: torch.Tensor            # pinned host uint8 H x W (original or marked)
    payload: torch.Tensor | None = None   # encode: packed message (pinned host)
    nbits: int = 0                 # encode: message bits; decode: bits to extract
    b: int = 0                     # decode: the public b
    lmr_map: torch.Tensor | None = None   # LMR decode: packed rotated map (pinned host)
    lmr_eta: torch.Tensor | None = None
    arrival: float = 0.0           # seconds on the server clock
    done: float = -1.0
    result: dict = field(default_factory=dict)

    @property
    def pixels(self) -> int:
        return int(self.image.numel())

    def device_bytes(self) -> int:
        """Device memory the request holds while in flight (buffers + workspace share)."""
        N = self.pixels
        words = ((N + 31) // 32) * 4
        msg = ((self.nbits + 31) // 32) * 4 + 4
        return 4 * N + 2 * words + 2 * msg + N + N // 4 + 4096


class PinnedPool:
    """Reusable pinned host buffers in power-of-two size classes.  Allocating pinned
    memory is a slow driver call; a serving loop that hands results back through
    pinned buffers recycles them once the caller has consumed a result."""

    def __init__(self):
        self.free: dict[int, list[torch.Tensor]] = {}

    @staticmethod
    def _cls(nbytes: int) -> int:
        return max(4096, 1 << (max(int(nbytes), 1) - 1).bit_length())

    def take(self, shape) -> torch.Tensor:
        nbytes = int(np.prod(shape)) if len(shape) else 1
        c = self._cls(nbytes)
        lst = self.free.get(c)
        buf = lst.pop() if lst else torch.empty(c, dtype=torch.uint8, pin_memory=True)
        return buf[:nbytes].view(*shape)

    def give(self, t: torch.Tensor):
        base = t._base if t._base is not None else t
        self.free.setdefault(base.numel(), []).append(base)


class _Batch:
    def __init__(self, reqs, stream):
        self.reqs = reqs
        self.stream = stream
        self.event = torch.cuda.Event()
        self.keep = []          # device tensors and plans alive until completion


class Server:
    def __init__(self, budget_bytes: float = 40e9, max_batch: int = 64, max_batch_pixels: int = 1 << 27,
                 streams: int = 4, device: int = 0, pool: "PinnedPool | None" = None):
        self.budget = float(budget_bytes)
        self.max_batch = max_batch
        self.max_batch_pixels = max_batch_pixels
        self.device = torch.device("cuda", device)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(streams)]
        self.free_streams = deque(self.streams)
        self.in_use = 0.0
        self.inflight: list[_Batch] = []
        self.queue: deque[Request] = deque()
        self.completed: list[Request] = []
        self.pool = pool if pool is not None else PinnedPool()
        self.consume = None
        self.t0 = None

    def now(self) -> float:
        return time.perf_counter() - self.t0

    # ------------------------------------------------------------------ launch --
    def _launch(self, reqs: list[Request]):
        st = self.free_streams.popleft()
        bt = _Batch(reqs, st)
        dev = self.device
        with torch.cuda.stream(st):
            info = rd.new_info(len(reqs), dev)
            bt.keep.append(info)
            if reqs[0].kind == "encode":
                self._launch_encode(bt, reqs, info, st, dev)
            else:
                self._launch_decode(bt, reqs, info, st, dev)
            bt.event.record(st)
        self.inflight.append(bt)

    def _launch_encode(self, bt, reqs, info, st, dev):
        # buffers and plans first (a plan upload waits for its stream), then copies and work
        imgs = [torch.empty(r.image.shape, dtype=torch.uint8, device=dev) for r in reqs]
        enc = [torch.empty_like(x) for x in imgs]
        marked = [torch.empty_like(x) for x in imgs]
        lmr = [(r.params.variant & 1) == rd.LMR for r in reqs]
        maps = [rd.bitbuf(x.numel(), dev) if l else None for x, l in zip(imgs, lmr)]
        etas = [rd.bitbuf(x.numel(), dev) if l else None for x, l in zip(imgs, lmr)]
        pays = [rd.bitbuf(r.nbits, dev) for r in reqs]
        j1 = [rd.make_job(r.params, *r.image.shape, src=imgs[i], dst=enc[i], map_bits=maps[i], eta_bits=etas[i],
                          info=info[i]) for i, r in enumerate(reqs)]
        j2 = [rd.make_job(r.params, *r.image.shape, src=enc[i], dst=marked[i], map_bits=maps[i], payload=pays[i],
                          nbits=r.nbits, info=info[i], b=0) for i, r in enumerate(reqs)]
        p1, p2 = rd.Plan(j1, st), rd.Plan(j2, st)
        for i, r in enumerate(reqs):
            imgs[i].copy_(r.image, non_blocking=True)
            pays[i][: r.payload.numel()].copy_(r.payload, non_blocking=True)
        p1.run(rd.OP_LABEL_ENCRYPT, st)
        p2.run(rd.OP_EMBED, st)
        outs = []
        for i, r in enumerate(reqs):
            h = self.pool.take(tuple(r.image.shape))
            h.copy_(marked[i], non_blocking=True)
            o = {"marked": h}
            if lmr[i]:
                hm = self.pool.take(tuple(maps[i].shape))
                he = self.pool.take(tuple(etas[i].shape))
                hm.copy_(maps[i], non_blocking=True)
                he.copy_(etas[i], non_blocking=True)
                o.update(map_bits=hm, eta_bits=he)
            outs.append(o)
        hinfo = self.pool.take(tuple(info.shape))
        hinfo.copy_(info, non_blocking=True)
        bt.keep += [imgs, enc, marked, maps, etas, pays, p1, p2]
        bt.outs, bt.hinfo = outs, hinfo

    def _launch_decode(self, bt, reqs, info, st, dev):
        imgs = [torch.empty(r.image.shape, dtype=torch.uint8, device=dev) for r in reqs]
        rec = [torch.empty_like(x) for x in imgs]
        maps = [torch.empty(r.lmr_map.shape, dtype=torch.uint8, device=dev) if r.lmr_map is not None else None
                for r in reqs]
        etas = [torch.empty(r.lmr_eta.shape, dtype=torch.uint8, device=dev) if r.lmr_eta is not None else None
                for r in reqs]
        bits = [rd.bitbuf(r.nbits, dev) for r in reqs]
        j1 = [rd.make_job(r.params, *r.image.shape, src=imgs[i], map_bits=maps[i], bits_out=bits[i], max_bits=r.nbits,
                          info=info[i], b=r.b) for i, r in enumerate(reqs)]
        j2 = [rd.make_job(r.params, *r.image.shape, src=imgs[i], dst=rec[i], map_bits=maps[i], eta_bits=etas[i],
                          info=info[i], b=r.b) for i, r in enumerate(reqs)]
        p1, p2 = rd.Plan(j1, st), rd.Plan(j2, st)
        for i, r in enumerate(reqs):
            imgs[i].copy_(r.image, non_blocking=True)
            if maps[i] is not None:
                maps[i].copy_(r.lmr_map, non_blocking=True)
                etas[i].copy_(r.lmr_eta, non_blocking=True)
        p1.run(rd.OP_EXTRACT, st)
        p2.run(rd.OP_DECRYPT_RECOVER, st)
        outs = []
        for i, r in enumerate(reqs):
            hb = self.pool.take(tuple(bits[i].shape))
            hr = self.pool.take(tuple(r.image.shape))
            hb.copy_(bits[i], non_blocking=True)
            hr.copy_(rec[i], non_blocking=True)
            outs.append({"bits": hb, "recovered": hr})
        hinfo = self.pool.take(tuple(info.shape))
        hinfo.copy_(info, non_blocking=True)
        bt.keep += [imgs, rec, maps, etas, bits, p1, p2]
        bt.outs, bt.hinfo = outs, hinfo

    # -------------------------------------------------------------------- loop --
    def _retire(self, block=False):
        still = []
        for bt in self.inflight:
            if block or bt.event.query():
                bt.event.synchronize()
                t = self.now()
                infos = rd.read_info(bt.hinfo)
                self.pool.give(bt.hinfo)
                for r, o, inf in zip(bt.reqs, bt.outs, infos):
                    r.result = {**o, "info": inf}
                    r.done = t
                    self.in_use -= r.device_bytes()
                    self.completed.append(r)
                    if self.consume is not None:
                        self.consume(r)
                self.free_streams.append(bt.stream)
                block = False
            else:
                still.append(bt)
        self.inflight = still

    def _admit_batch(self) -> list[Request]:
        """Up to max_batch same-kind requests from the head of the queue that fit."""
        if not self.queue or not self.free_streams:
            return []
        kind = self.queue[0].kind
        batch, px = [], 0
        while self.queue and len(batch) < self.max_batch:
            r = self.queue[0]
            if r.kind != kind or px + r.pixels > self.max_batch_pixels and batch:
                break
            need = r.device_bytes()
            if self.in_use + need > self.budget and (batch or self.inflight):
                break
            self.queue.popleft()
            self.in_use += need
            batch.append(r)
            px += r.pixels
        return batch

    def release(self, r: Request):
        """Give a completed request's pinned result buffers back for reuse; the result
        tensors must not be read afterwards."""
        for v in list(r.result.values()):
            if isinstance(v, torch.Tensor) and v.is_pinned():
                self.pool.give(v)
        r.result = {"info": r.result.get("info")}

    def run(self, requests: list[Request], realtime: bool = True, consume=None) -> list[Request]:
        """Serve requests whose `arrival` is on the server clock (seconds from start).
        realtime=False admits everything at once (arrival times ignored).  consume(r),
        if given, is called as each request completes (e.g. to hand the result on and
        release its buffers)."""
        self.consume = consume
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        self.t0 = time.perf_counter()
        if not realtime:
            for r in pending:
                r.arrival = 0.0
        while pending or self.queue or self.inflight:
            now = self.now()
            while pending and pending[0].arrival <= now:
                self.queue.append(pending.popleft())
            self._retire()
            launched = False
            while True:
                b = self._admit_batch()
                if not b:
                    break
                self._launch(b)
                launched = True
            if not launched and not self.queue and self.inflight and pending:
                # idle until the next arrival or a completion
                time.sleep(max(0.0, min(pending[0].arrival - self.now(), 2e-4)))
            elif not launched and self.inflight and not self.free_streams:
                self._retire(block=True)
        return self.completed


def latency_stats(done: list[Request]) -> dict:
    lat = np.array([r.done - r.arrival for r in done]) * 1e3
    px = sum(r.pixels for r in done)
    span = max(r.done for r in done) - min(r.arrival for r in done)
    return {"requests": len(done), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "sustained_mpx": px / span / 1e6 if span > 0 else None}
