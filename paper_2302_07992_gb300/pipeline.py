"""Batched pipelines over the C ABI: a fixed set of images (any sizes, both variants)
with their device buffers and the four plans, run eagerly or replayed as one captured
CUDA graph, plus the per-image form (one plan per image and operation) it is compared
against.  Argument marshalling and buffer management only -- all work is in the
library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import rdhei as rd
from . import synth

OPS = (rd.OP_LABEL_ENCRYPT, rd.OP_EMBED, rd.OP_EXTRACT, rd.OP_DECRYPT_RECOVER)


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
        return rd.make_job(p, H, W, src=self.marked[i], dst=self.rec[i], map_bits=self.maps[i],
                           eta_bits=self.etas[i], info=self.info[i], b=0)

    def pixels(self) -> int:
        return sum(H * W for H, W in self.shapes)


class BatchedPipeline:
    """One plan per operation over the whole set; a step is four plan runs, optionally
    captured into a single CUDA graph."""

    def __init__(self, s: ImageSet, payload_fn, stream=None):
        self.s = s
        stream = stream or torch.cuda.current_stream()
        enc = rd.Plan(s.encode_jobs(), stream)
        enc.run(rd.OP_LABEL_ENCRYPT, stream)
        torch.cuda.synchronize()
        s.set_payloads(payload_fn)
        self.plans = [(enc, rd.OP_LABEL_ENCRYPT)]
        for op in OPS[1:]:
            self.plans.append((rd.Plan([s.job(op, i) for i in range(s.n)], stream), op))
        self.graph = None

    def step(self, stream=None):
        for pl, op in self.plans:
            pl.run(op, stream)

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
    """The plain form: every image runs its own four single-image plans."""

    def __init__(self, s: ImageSet, stream=None):
        self.s = s
        stream = stream or torch.cuda.current_stream()
        self.plans = [[(rd.Plan([s.job(op, i)], stream), op) for op in OPS] for i in range(s.n)]

    def step(self, stream=None):
        for per in self.plans:
            for pl, op in per:
                pl.run(op, stream)

    def launches_per_step(self) -> int:
        return sum(len(pl.active_stages(op)) for per in self.plans for pl, op in per)


def default_payload(seed_of):
    return lambda i, nbits: synth.payload_bits(seed_of(i), nbits)
