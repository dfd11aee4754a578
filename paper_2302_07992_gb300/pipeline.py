"""Batched pipelines over the C ABI: a fixed set of images (any sizes, both variants)
with their device buffers and one plan per operation, run eagerly or replayed as one
captured CUDA graph, plus the per-image form (one plan per image and operation) it is
compared against.  A round trip is either the four separable calls of the paper's
parties or the two fused ones (rdhei_encode: owner + hider; rdhei_decode: receiver with
both keys).  Argument marshalling and buffer management only -- all work is in the
library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import rdhei as rd
from . import synth

OPS = (rd.OP_LABEL_ENCRYPT, rd.OP_EMBED, rd.OP_EXTRACT, rd.OP_DECRYPT_RECOVER)
FUSED_OPS = (rd.OP_ENCODE, rd.OP_DECODE)


class ImageSet:
    """Device buffers of one encode + decode round trip for each image."""

    def __init__(self, imgs, variants, params, side_bits=None, device="cuda"):
        self.n = len(imgs)
        self.variants = list(variants)
        self.params = list(params)
        self.shapes = [tuple(im.shape) for im in imgs]
        self.img = [torch.as_tensor(np.ascontiguousarray(im)).to(device) for im in imgs]
        self.enc = [torch.empty_like(x) for x in self.img]
        self.marked = [torch.empty_like(x) for x in self.img]
        self.rec = [torch.empty_like(x) for x in self.img]
        N = [x.numel() for x in self.img]
        lmr = [(v & 1) == rd.LMR for v in self.variants]
        self.maps = [rd.bitbuf(N[i], device) if lmr[i] else None for i in range(self.n)]
        self.etas = [rd.bitbuf(N[i], device) if lmr[i] else None for i in range(self.n)]
        self.side_n = [0] * self.n
        self.side = [None] * self.n
        if side_bits is not None:
            for i in range(self.n):
                if lmr[i] and side_bits[i] is not None:
                    nbits, packed = side_bits[i]
                    self.side_n[i] = int(nbits)
                    self.side[i] = rd.as_bitbuf(torch.as_tensor(packed), nbits)
        self.info = rd.new_info(self.n, device)
        self.caps = None
        self.payload = [None] * self.n
        self.bits = [None] * self.n

    def encode_jobs(self):
        return [rd.make_job(self.params[i], *self.shapes[i], src=self.img[i], dst=self.enc[i], map_bits=self.maps[i],
                            eta_bits=self.etas[i], side_bits=self.side[i], side_nbits=self.side_n[i],
                            info=self.info[i]) for i in range(self.n)]

    def set_payloads(self, payload_fn):
        """After one label_encrypt: full-capacity payloads (payload_fn(i, nbits) -> packed bytes)."""
        self.caps = [r["capacity"] for r in rd.read_info(self.info)]
        for i in range(self.n):
            self.payload[i] = rd.as_bitbuf(torch.as_tensor(payload_fn(i, self.caps[i])), self.caps[i])
            self.bits[i] = rd.bitbuf(self.caps[i], self.img[i].device)

    def job(self, op, i):
        p, (H, W) = self.params[i], self.shapes[i]
        if op == rd.OP_LABEL_ENCRYPT:
            return self.encode_jobs()[i]
        if op == rd.OP_EMBED:
            return rd.make_job(p, H, W, src=self.enc[i], dst=self.marked[i], map_bits=self.maps[i],
                               payload=self.payload[i], nbits=self.caps[i], info=self.info[i], b=0)
        if op == rd.OP_EXTRACT:
            return rd.make_job(p, H, W, src=self.marked[i], map_bits=self.maps[i], bits_out=self.bits[i],
                               max_bits=self.caps[i], info=self.info[i], b=0)
        if op == rd.OP_ENCODE:
            return rd.make_job(p, H, W, src=self.img[i], dst=self.marked[i], map_bits=self.maps[i],
                               eta_bits=self.etas[i], side_bits=self.side[i], side_nbits=self.side_n[i],
                               payload=self.payload[i], nbits=self.caps[i], info=self.info[i])
        if op == rd.OP_DECODE:
            return rd.make_job(p, H, W, src=self.marked[i], dst=self.rec[i], map_bits=self.maps[i],
                               eta_bits=self.etas[i], bits_out=self.bits[i], max_bits=self.caps[i],
                               info=self.info[i], b=0)
        return rd.make_job(p, H, W, src=self.marked[i], dst=self.rec[i], map_bits=self.maps[i],
                           eta_bits=self.etas[i], info=self.info[i], b=0)

    def pixels(self) -> int:
        return sum(H * W for H, W in self.shapes)


class BatchedPipeline:
    """One plan per operation over the whole set; a step is four plan runs (two with
    fused=True), optionally captured into a single CUDA graph."""

    def __init__(self, s: ImageSet, payload_fn, stream=None, fused: bool = False):
        self.s = s
        stream = stream or torch.cuda.current_stream()
        enc = rd.Plan(s.encode_jobs(), stream)
        enc.run(rd.OP_LABEL_ENCRYPT, stream)        # the capacities size the payloads
        torch.cuda.synchronize()
        s.set_payloads(payload_fn)
        if fused:
            self.plans = [(rd.Plan([s.job(op, i) for i in range(s.n)], stream), op) for op in FUSED_OPS]
        else:
            self.plans = [(enc, rd.OP_LABEL_ENCRYPT)]
            for op in OPS[1:]:
                self.plans.append((rd.Plan([s.job(op, i) for i in range(s.n)], stream), op))
        self.graph = None

    def step(self, stream=None):
        for pl, op in self.plans:
            pl.run(op, stream)

    def plan(self, op):
        return next(pl for pl, o in self.plans if o == op)

    def jobs(self, op):
        return [self.s.job(op, i) for i in range(self.s.n)]

    def capture(self):
        """Record one step into a CUDA graph (plans issue memsets and kernels only)."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.step(side)                      # warm the launch path outside capture
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step(torch.cuda.current_stream())
        return self.graph

    def replay(self):
        self.graph.replay()

    def launches_per_step(self) -> int:
        return sum(len(pl.active_stages(op)) for pl, op in self.plans)


class PerImagePipeline:
    """The plain form: every image runs its own single-image plans (four, or two with
    fused=True)."""

    def __init__(self, s: ImageSet, stream=None, fused: bool = False):
        self.s = s
        stream = stream or torch.cuda.current_stream()
        ops = FUSED_OPS if fused else OPS
        self.plans = [[(rd.Plan([s.job(op, i)], stream), op) for op in ops] for i in range(s.n)]

    def step(self, stream=None):
        for per in self.plans:
            for pl, op in per:
                pl.run(op, stream)

    def launches_per_step(self) -> int:
        return sum(len(pl.active_stages(op)) for per in self.plans for pl, op in per)


def default_payload(seed_of):
    return lambda i, nbits: synth.payload_bits(seed_of(i), nbits)


class OverlappedPipeline:
    """Host-to-host processing of a batch of equal-size images with the copies hidden
    behind the kernels.  The batch is cut into chunks; each chunk has its own four
    plans.  Chunk c's inputs (pixels, payload bits, LMR side bits) go up on an upload
    stream while chunk c - 1 runs the four operations on the compute stream and chunk
    c - 2's results (recovered pixels, extracted bits) come down on a download stream.
    Events order the reuse of each chunk's device buffers from one run to the next.
    Payloads and extracted bits are packed per image to their capacity, so only the
    bytes that carry bits cross the bus.  fused=True runs rdhei_encode and rdhei_decode
    per chunk instead of the four separable calls."""

    def __init__(self, n, H, W, variants, params, caps, side_nbits=None, chunks=4, device="cuda", wave_cols=None,
                 graphs=True, fused: bool = False):
        self.n, self.H, self.W = n, H, W
        self.dev = torch.device(device)
        N = H * W
        self.variants = list(variants)
        lmr = [(v & 1) == rd.LMR for v in self.variants]
        self.caps = [int(c) for c in caps]
        # per-image offsets into the packed payload / bits buffers (16-byte aligned)
        self.pay_off, off = [], 0
        for c in self.caps:
            self.pay_off.append(off)
            off += ((c + 127) // 128) * 16
        self.pay_bytes = max(off, 16)
        self.side_nbits = [int(side_nbits[i]) if (side_nbits is not None and lmr[i]) else 0 for i in range(n)]
        self.side_off, off = [], 0
        for s in self.side_nbits:
            self.side_off.append(off)
            off += ((s + 127) // 128) * 16
        self.side_bytes = max(off, 16)
        dev = self.dev
        self.img = torch.empty((n, H, W), dtype=torch.uint8, device=dev)
        self.enc = torch.empty_like(self.img)
        self.marked = torch.empty_like(self.img)
        self.rec = torch.empty_like(self.img)
        mb = ((N + 31) // 32) * 4
        self.maps = torch.zeros((n, mb), dtype=torch.uint8, device=dev)
        self.etas = torch.zeros((n, mb), dtype=torch.uint8, device=dev)
        self.pay = torch.zeros(self.pay_bytes, dtype=torch.uint8, device=dev)
        self.bits = torch.zeros(self.pay_bytes, dtype=torch.uint8, device=dev)
        self.side = torch.zeros(self.side_bytes, dtype=torch.uint8, device=dev)
        self.info = rd.new_info(n, dev)
        self.up, self.comp, self.down = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        bounds = np.linspace(0, n, chunks + 1).astype(int)
        self.chunks = [(int(a), int(b)) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
        self.plans = []
        for a, b in self.chunks:
            enc, emb, ext, dec = [], [], [], []
            for k in range(a, b):
                p = params[k]
                m = self.maps[k] if lmr[k] else None
                pay = self.pay[self.pay_off[k]:]
                bo = self.bits[self.pay_off[k]:]
                sd = self.side[self.side_off[k]:] if self.side_nbits[k] else None
                enc.append(rd.make_job(p, H, W, src=self.img[k], dst=self.enc[k], map_bits=m,
                                       eta_bits=self.etas[k] if lmr[k] else None, side_bits=sd,
                                       side_nbits=self.side_nbits[k], info=self.info[k]))
                emb.append(rd.make_job(p, H, W, src=self.enc[k], dst=self.marked[k], map_bits=m, payload=pay,
                                       nbits=self.caps[k], info=self.info[k], b=0))
                ext.append(rd.make_job(p, H, W, src=self.marked[k], map_bits=m, bits_out=bo, max_bits=self.caps[k],
                                       info=self.info[k], b=0))
                dec.append(rd.make_job(p, H, W, src=self.marked[k], dst=self.rec[k], map_bits=m,
                                       eta_bits=self.etas[k] if lmr[k] else None, info=self.info[k], b=0))
            if fused:
                fenc = [rd.make_job(params[k], H, W, src=self.img[k], dst=self.marked[k],
                                    map_bits=self.maps[k] if lmr[k] else None,
                                    eta_bits=self.etas[k] if lmr[k] else None,
                                    side_bits=self.side[self.side_off[k]:] if self.side_nbits[k] else None,
                                    side_nbits=self.side_nbits[k], payload=self.pay[self.pay_off[k]:],
                                    nbits=self.caps[k], info=self.info[k]) for k in range(a, b)]
                fdec = [rd.make_job(params[k], H, W, src=self.marked[k], dst=self.rec[k],
                                    map_bits=self.maps[k] if lmr[k] else None,
                                    eta_bits=self.etas[k] if lmr[k] else None, bits_out=self.bits[self.pay_off[k]:],
                                    max_bits=self.caps[k], info=self.info[k], b=0) for k in range(a, b)]
                self.plans.append([(rd.Plan(fenc, self.comp), rd.OP_ENCODE),
                                   (rd.Plan(fdec, self.comp, wave_cols=wave_cols), rd.OP_DECODE)])
                continue
            self.plans.append([(rd.Plan(enc, self.comp), rd.OP_LABEL_ENCRYPT), (rd.Plan(emb, self.comp), rd.OP_EMBED),
                               (rd.Plan(ext, self.comp), rd.OP_EXTRACT),
                               (rd.Plan(dec, self.comp, wave_cols=wave_cols), rd.OP_DECRYPT_RECOVER)])
        nc = len(self.chunks)
        self.ev_comp = [torch.cuda.Event() for _ in range(nc)]
        self.ev_down = [torch.cuda.Event() for _ in range(nc)]
        self.started = False
        # each chunk's four operations as one CUDA graph (fewer launch gaps on the GPU)
        self.graphs = None
        if graphs:
            with torch.cuda.stream(self.comp):
                for per in self.plans:
                    for plan, op in per:
                        plan.run(op, self.comp)          # warm the launch path outside capture
            self.comp.synchronize()
            self.graphs = []
            for per in self.plans:
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=self.comp):
                    for plan, op in per:
                        plan.run(op, self.comp)
                self.graphs.append(g)

    def host_buffers(self):
        """Pinned host buffers of the right sizes: (pixels, payload, side) in and
        (recovered, bits) out."""
        n, H, W = self.n, self.H, self.W
        pin = dict(dtype=torch.uint8, pin_memory=True)
        return (torch.empty((n, H, W), **pin), torch.zeros(self.pay_bytes, **pin), torch.zeros(self.side_bytes, **pin),
                torch.empty((n, H, W), **pin), torch.zeros(self.pay_bytes, **pin))

    def pack_payloads(self, h_pay, payloads):
        for k, p in enumerate(payloads):
            nb = (self.caps[k] + 7) // 8
            h_pay[self.pay_off[k]:self.pay_off[k] + nb].copy_(torch.as_tensor(np.asarray(p, np.uint8)[:nb]))

    def pack_side(self, h_side, sides):
        for k, s in enumerate(sides):
            if self.side_nbits[k]:
                nb = (self.side_nbits[k] + 7) // 8
                h_side[self.side_off[k]:self.side_off[k] + nb].copy_(torch.as_tensor(np.asarray(s, np.uint8)[:nb]))

    def _span(self, offs, sizes, a, b):
        lo = offs[a]
        hi = offs[b - 1] + ((sizes[b - 1] + 127) // 128) * 16
        return lo, hi

    def run(self, h_img, h_pay, h_side, h_rec, h_bits):
        """Enqueue one host-to-host pass over the batch; returns the download stream
        (synchronise on it, or record an event)."""
        for c, (a, b) in enumerate(self.chunks):
            pl, ph = self._span(self.pay_off, self.caps, a, b)
            sl, sh = self._span(self.side_off, self.side_nbits, a, b)
            with torch.cuda.stream(self.up):
                if self.started:
                    self.up.wait_event(self.ev_comp[c])       # the previous run's kernels read these buffers
                self.img[a:b].copy_(h_img[a:b], non_blocking=True)
                if ph > pl:
                    self.pay[pl:ph].copy_(h_pay[pl:ph], non_blocking=True)
                if sh > sl:
                    self.side[sl:sh].copy_(h_side[sl:sh], non_blocking=True)
                up_done = torch.cuda.Event()
                up_done.record(self.up)
            self.comp.wait_event(up_done)
            if self.started:
                self.comp.wait_event(self.ev_down[c])         # results of the previous run are down
            if self.graphs is not None:
                with torch.cuda.stream(self.comp):
                    self.graphs[c].replay()
            else:
                for plan, op in self.plans[c]:
                    plan.run(op, self.comp)
            self.ev_comp[c].record(self.comp)
            with torch.cuda.stream(self.down):
                self.down.wait_event(self.ev_comp[c])
                h_rec[a:b].copy_(self.rec[a:b], non_blocking=True)
                if ph > pl:
                    h_bits[pl:ph].copy_(self.bits[pl:ph], non_blocking=True)
                self.ev_down[c].record(self.down)
        self.started = True
        return self.down

    def status(self) -> int:
        codes = [pl.status(self.comp) for per in self.plans for pl, _ in per]
        return max(codes) if codes else 0
