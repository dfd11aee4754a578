"""Continuous-batching request loop for encode and decode requests on one GPU.

  encode request: an original image and a message -> rdhei_encode (owner + hider)
                  -> marked image (and, for LMR, the rotated maps);
  decode request: a marked image (+ LMR maps) -> rdhei_decode (receiver with both keys)
                  -> message bits and recovered image.
(CudaExecutor(fused=False) runs the four separable calls instead.)

Device-resident state: an encode request with keep_state leaves its rotated LMR maps
(map l and first-MSB map eta, 2 bits a pixel) in device memory and returns a handle; a
decode request that names the handle reads them there, so they never cross the host
link.  The store (DeviceState) is charged to the admission budget and evicts the
least recently used entries beyond its own cap.

Admission, batching, cancellation, failure handling and metrics are the device-free
scheduler of ``sched``; this module supplies its CUDA executor.  Each admitted group
of same-kind requests becomes one batch: one plan over all its images, its descriptors
uploaded asynchronously from a pinned staging buffer, launched on its own stream, with
host<->device copies on that stream -- nothing in a launch waits for the device.  New batches
are formed and launched while earlier ones run, so work of requests that arrive while
others are on the GPU overlaps on the device.  A request's latency is arrival -> its
batch's completion (results back in host memory).  All work is in the library's
kernels; this module marshals buffers, plans and streams.  Each launch is an NVTX
range ("serve.encode[n]" / "serve.decode[n]"), around the library's own per-call
ranges.
"""
from __future__ import annotations

import math
from collections import OrderedDict, deque

import torch

from . import rdhei as rd
from .sched import LAT_EDGES_MS, STATUSES, Request, Scheduler, latency_stats  # noqa: F401


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
        nbytes = math.prod(int(x) for x in shape) if len(shape) else 1
        c = self._cls(nbytes)
        lst = self.free.get(c)
        buf = lst.pop() if lst else torch.empty(c, dtype=torch.uint8, pin_memory=True)
        return buf[:nbytes].view(*shape)

    def give(self, t: torch.Tensor):
        base = t._base if t._base is not None else t
        self.free.setdefault(base.numel(), []).append(base)


class DeviceState:
    """Per-image LMR maps kept in device memory between an encode and later decodes of
    the same image, under a byte cap (least recently used entries are evicted)."""

    def __init__(self, cap_bytes: float = 4e9):
        self.cap = float(cap_bytes)
        self.items: OrderedDict[int, torch.Tensor] = OrderedDict()
        self.bytes = 0
        self._next = 1

    def put(self, buf: torch.Tensor) -> int:
        h = self._next
        self._next += 1
        self.items[h] = buf
        self.bytes += buf.numel()
        while self.bytes > self.cap and len(self.items) > 1:
            _, old = self.items.popitem(last=False)
            self.bytes -= old.numel()
        return h

    def get(self, handle: int) -> torch.Tensor | None:
        buf = self.items.get(handle)
        if buf is not None:
            self.items.move_to_end(handle)
        return buf

    def drop(self, handle: int):
        buf = self.items.pop(handle, None)
        if buf is not None:
            self.bytes -= buf.numel()


class _Batch:
    def __init__(self, reqs, stream):
        self.reqs = reqs
        self.stream = stream
        self.event = torch.cuda.Event()
        self.keep = []          # device tensors and plans alive until completion
        self.plans = []
        self.outs, self.hinfo, self.hcodes = None, None, None


class CudaExecutor:
    """Runs a scheduler batch on the GPU: one stream per batch in flight, one plan per
    operation, pinned result buffers from a PinnedPool."""

    def __init__(self, streams: int = 4, device: int = 0, pool: "PinnedPool | None" = None,
                 state: "DeviceState | None" = None, fused: bool = True):
        self.fused = fused
        self.device = torch.device("cuda", device)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(streams)]
        self.free_streams = deque(self.streams)
        self.slots = streams
        self.pool = pool if pool is not None else PinnedPool()
        self.state = state if state is not None else DeviceState()
        # per stream and kind, the device arena of its last batch, reused while large enough
        # (a stream takes a new batch only after the previous one completed); each holds at
        # most twice the largest batch that stream has run
        self._arenas: dict = {}

    def state_bytes(self) -> int:
        return self.state.bytes

    def launch(self, reqs: list[Request]) -> _Batch:
        st = self.free_streams.popleft()
        bt = _Batch(reqs, st)
        dev = self.device
        torch.cuda.nvtx.range_push(f"serve.{reqs[0].kind}[{len(reqs)}]")
        try:
            with torch.cuda.stream(st):
                if reqs[0].kind == "encode":
                    self._launch_encode(bt, reqs, st, dev)
                else:
                    self._launch_decode(bt, reqs, st, dev)
                bt.event.record(st)
        except Exception:
            st.synchronize()                    # nothing of this batch may still use its buffers
            self.free_streams.append(st)
            raise
        finally:
            torch.cuda.nvtx.range_pop()
        return bt

    def ready(self, bt: _Batch) -> bool:
        return bt.event.query()

    def wait(self, bt: _Batch):
        bt.event.synchronize()

    def results(self, bt: _Batch) -> list[dict]:
        n = len(bt.outs)
        infos = rd.read_info(bt.hinfo[: n * rd.INFO_BYTES].view(n, rd.INFO_BYTES))
        # the plans' workspace error words came down behind the infos, in the same copy: a
        # device-side failure (timeout, index check) fails the whole batch; ECAPACITY is a
        # per-request outcome
        codes = bt.hinfo[n * rd.INFO_BYTES:].view(torch.int32)[: bt.hcodes].tolist()
        self.pool.give(bt.hinfo)
        bt.hinfo, bt.hcodes = None, None
        for code in codes:
            if code not in (0, rd.RDHEI_ECAPACITY):
                for o in bt.outs:
                    self.discard(o)
                raise rd.RdheiError(f"device reported {rd.STATUS.get(code, code)}")
        return [{**o, "info": inf} for o, inf in zip(bt.outs, infos)]

    def _infos_down(self, bt: _Batch, info_err: torch.Tensor, n: int, plans, st):
        """The plans' error words into the device words behind the n infos, then one copy
        of both into pinned memory, read once the batch's event fired."""
        err = info_err[n * rd.INFO_BYTES:].view(torch.int32)
        for i, pl in enumerate(plans):
            pl.copy_status(err[i:i + 1], st)
        hinfo = self.pool.take((info_err.numel(),))
        hinfo.copy_(info_err, non_blocking=True)
        bt.hinfo, bt.hcodes = hinfo, len(plans)

    def discard(self, result: dict, drop_state: bool = True):
        """Give back a result's pinned buffers; unless drop_state is False, also its
        device-resident maps (a result nobody will read)."""
        for v in result.values():
            if isinstance(v, torch.Tensor):          # result tensors all come from the pool
                self.pool.give(v)
        if drop_state and result.get("state"):
            self.state.drop(result["state"])

    def release(self, bt: _Batch):
        for pl in bt.plans:
            if getattr(pl, "staging", None) is not None:
                self.pool.give(pl.staging)          # the upload is long done: the batch completed
                pl.staging = None
        bt.keep.clear()
        bt.plans.clear()
        self.free_streams.append(bt.stream)

    def _plan(self, jobs, st):
        return rd.Plan(jobs, st, staging=lambda nb: self.pool.take((nb,)))

    def _arena(self, sizes, zero: bool, dev, key=None):
        """Device memory cut into 256-byte-aligned pieces of the given sizes (None for a
        size of None), zero-filled when the kernels OR into it.  With a key, the arena of
        the key's previous batch is reused when large enough, else replaced by one of the
        next power-of-two size."""
        offs, tot = [], 0
        for n in sizes:
            offs.append(None if n is None else tot)
            if n is not None:
                tot += (int(n) + 255) & ~255
        tot = max(tot, 256)
        buf = self._arenas.get(key) if key is not None else None
        if buf is None or buf.numel() < tot:
            size = 1 << (tot - 1).bit_length() if key is not None else tot
            buf = torch.empty(size, dtype=torch.uint8, device=dev)
            if key is not None:
                self._arenas[key] = buf
        if zero:
            buf[:tot].zero_()
        return buf, [None if o is None else buf[o:o + int(n)] for o, n in zip(offs, sizes)]

    @staticmethod
    def _words(nbits: int) -> int:
        return max(4, ((int(nbits) + 31) // 32) * 4)

    def _launch_encode(self, bt, reqs, st, dev):
        # buffers and plans first, then copies and work, all on the batch's stream
        n = len(reqs)
        px = [r.pixels for r in reqs]
        lmr = [(r.params.variant & 1) == rd.LMR for r in reqs]
        img_arena, views = self._arena(px * (2 if self.fused else 3), False, dev, (st.cuda_stream, "img"))
        imgs = [v.view(*r.image.shape) for v, r in zip(views[:n], reqs)]
        marked = [v.view(*r.image.shape) for v, r in zip(views[n:2 * n], reqs)]
        enc = [v.view(*r.image.shape) for v, r in zip(views[2 * n:], reqs)]     # separable calls only
        keep = [l and r.keep_state for l, r in zip(lmr, reqs)]
        bit_arena, bviews = self._arena([self._words(p) if l and not k else None for p, l, k in zip(px, lmr, keep)]
                                        * 2 + [self._words(r.nbits) for r in reqs] + [n * rd.INFO_BYTES + 16], True,
                                        dev, (st.cuda_stream, "bits"))
        maps, etas, pays = bviews[:n], bviews[n:2 * n], bviews[2 * n:3 * n]
        info = bviews[-1][: n * rd.INFO_BYTES].view(n, rd.INFO_BYTES)
        # maps that stay on the device get an allocation of their own (the store holds it)
        kept = {}
        for i, r in enumerate(reqs):
            if keep[i]:
                w = self._words(px[i])
                buf = torch.empty(2 * w, dtype=torch.uint8, device=dev)
                maps[i], etas[i] = buf[:w], buf[w:]
                kept[i] = buf
        if self.fused:
            jf = [rd.make_job(r.params, *r.image.shape, src=imgs[i], dst=marked[i], map_bits=maps[i],
                              eta_bits=etas[i], payload=pays[i], nbits=r.nbits, info=info[i])
                  for i, r in enumerate(reqs)]
            plans = [(self._plan(jf, st), rd.OP_ENCODE)]
        else:
            j1 = [rd.make_job(r.params, *r.image.shape, src=imgs[i], dst=enc[i], map_bits=maps[i],
                              eta_bits=etas[i], info=info[i]) for i, r in enumerate(reqs)]
            j2 = [rd.make_job(r.params, *r.image.shape, src=enc[i], dst=marked[i], map_bits=maps[i],
                              payload=pays[i], nbits=r.nbits, info=info[i], b=0) for i, r in enumerate(reqs)]
            plans = [(self._plan(j1, st), rd.OP_LABEL_ENCRYPT), (self._plan(j2, st), rd.OP_EMBED)]
        for i, r in enumerate(reqs):
            imgs[i].copy_(r.image, non_blocking=True)
            pays[i][: r.payload.numel()].copy_(r.payload, non_blocking=True)
        for pl, op in plans:
            pl.run(op, st)
        outs = []
        for i, r in enumerate(reqs):
            h = self.pool.take(tuple(r.image.shape))
            h.copy_(marked[i], non_blocking=True)
            o = {"marked": h}
            if i in kept:
                o["state"] = self.state.put(kept[i])
            elif lmr[i]:
                hm = self.pool.take(tuple(maps[i].shape))
                he = self.pool.take(tuple(etas[i].shape))
                hm.copy_(maps[i], non_blocking=True)
                he.copy_(etas[i], non_blocking=True)
                o.update(map_bits=hm, eta_bits=he)
            outs.append(o)
        self._infos_down(bt, bviews[-1], n, [pl for pl, _ in plans], st)
        bt.keep += [img_arena, bit_arena]
        bt.plans = [pl for pl, _ in plans]
        bt.outs = outs

    def _launch_decode(self, bt, reqs, st, dev):
        n = len(reqs)
        px = [r.pixels for r in reqs]
        # device-resident maps of an earlier encode, else the request's host maps
        held = [self.state.get(r.state) if r.state else None for r in reqs]
        for r, h in zip(reqs, held):
            if r.state and h is None and r.lmr_map is None:
                raise KeyError(f"device state {r.state} is gone and the request carries no maps")
        img_arena, views = self._arena(px * 2 + [r.lmr_map.numel() if r.lmr_map is not None and h is None else None
                                                 for r, h in zip(reqs, held)]
                                       + [r.lmr_eta.numel() if r.lmr_eta is not None and h is None else None
                                          for r, h in zip(reqs, held)], False, dev, (st.cuda_stream, "img"))
        imgs = [v.view(*r.image.shape) for v, r in zip(views[:n], reqs)]
        rec = [v.view(*r.image.shape) for v, r in zip(views[n:2 * n], reqs)]
        maps, etas = views[2 * n:3 * n], views[3 * n:]
        for i, h in enumerate(held):
            if h is not None:
                w = h.numel() // 2
                maps[i], etas[i] = h[:w], h[w:]
                h.record_stream(st)                 # allocated on the encode's stream, read on this one
                bt.keep.append(h)                   # alive until the batch completes, even if evicted
        bit_arena, bviews = self._arena([self._words(r.nbits) for r in reqs] + [n * rd.INFO_BYTES + 16], True, dev,
                                        (st.cuda_stream, "bits"))
        bits, info = bviews[:n], bviews[-1][: n * rd.INFO_BYTES].view(n, rd.INFO_BYTES)
        if self.fused:
            jf = [rd.make_job(r.params, *r.image.shape, src=imgs[i], dst=rec[i], map_bits=maps[i], eta_bits=etas[i],
                              bits_out=bits[i], max_bits=r.nbits, info=info[i], b=r.b) for i, r in enumerate(reqs)]
            plans = [(self._plan(jf, st), rd.OP_DECODE)]
        else:
            j1 = [rd.make_job(r.params, *r.image.shape, src=imgs[i], map_bits=maps[i], bits_out=bits[i],
                              max_bits=r.nbits, info=info[i], b=r.b) for i, r in enumerate(reqs)]
            j2 = [rd.make_job(r.params, *r.image.shape, src=imgs[i], dst=rec[i], map_bits=maps[i],
                              eta_bits=etas[i], info=info[i], b=r.b) for i, r in enumerate(reqs)]
            plans = [(self._plan(j1, st), rd.OP_EXTRACT), (self._plan(j2, st), rd.OP_DECRYPT_RECOVER)]
        for i, r in enumerate(reqs):
            imgs[i].copy_(r.image, non_blocking=True)
            if maps[i] is not None and held[i] is None:
                maps[i].copy_(r.lmr_map.reshape(-1), non_blocking=True)
                etas[i].copy_(r.lmr_eta.reshape(-1), non_blocking=True)
        for pl, op in plans:
            pl.run(op, st)
        outs = []
        for i, r in enumerate(reqs):
            hb = self.pool.take(tuple(bits[i].shape))
            hr = self.pool.take(tuple(r.image.shape))
            hb.copy_(bits[i], non_blocking=True)
            hr.copy_(rec[i], non_blocking=True)
            outs.append({"bits": hb, "recovered": hr})
        self._infos_down(bt, bviews[-1], n, [pl for pl, _ in plans], st)
        bt.keep += [img_arena, bit_arena]
        bt.plans = [pl for pl, _ in plans]
        bt.outs = outs


class Server(Scheduler):
    """The scheduler driving a CudaExecutor (the serving loop on one GPU)."""

    def __init__(self, budget_bytes: float = 40e9, max_batch: int = 64, max_batch_pixels: int = 1 << 27,
                 streams: int = 4, device: int = 0, pool: "PinnedPool | None" = None,
                 max_queue: int | None = None, state: "DeviceState | None" = None, admit_window_ms: float = 0.0,
                 fused: bool = True):
        ex = CudaExecutor(streams, device, pool, state, fused)
        super().__init__(ex, budget_bytes, max_batch, max_batch_pixels, max_queue, admit_window_ms=admit_window_ms)
        self.pool = ex.pool
        self.state = ex.state

    def release(self, r: Request):
        """Give a completed request's pinned result buffers back for reuse; the result
        tensors must not be read afterwards.  Device-resident maps stay (their handle
        is kept in the result) until drop_state() or eviction."""
        self.ex.discard(r.result, drop_state=False)
        r.result = {"info": r.result.get("info"), "state": r.result.get("state", 0)}

    def drop_state(self, handle: int):
        self.state.drop(handle)
