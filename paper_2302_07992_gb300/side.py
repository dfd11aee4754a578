"""LMR with its side information carried in the first MSB plane (Sec. III-B-1 to
III-B-3): the content owner's fit loop, and the hider's / receiver's read-back.

Owner (``lmr_encode``), for a batch of device images:
  1. ``rdhei_label_encrypt`` with the optimal b: I_e without side bits, rot(l), rot(eta)
     and the label histogram on the device;
  2. rot(eta) and rot(l) to the host; ``rdhei_lmr_side_pack`` compresses both (host
     threads) into the container;
  3. images whose container does not fit into H W bits move to their next candidate b
     (decreasing (b - 1) zeros(b), ties to the smaller b): ``rdhei_label_encrypt``
     with that b forced gives its rot(l) -- I_e itself does not depend on b -- and the
     pack is retried; an image with no fitting b is a bad case (no payload);
  4. the containers go back to the device and ``rdhei_lmr_set_side`` writes them into
     bit 7 of I_e.
Hider / receiver (``lmr_read_side``): ``rdhei_msb_plane`` packs bit 7 of the device
image, the plane comes to the host, ``rdhei_lmr_side_unpack`` returns b, rot(eta) and
rot(l), which go back to the device for ``rdhei_embed`` / ``rdhei_extract`` /
``rdhei_decrypt_recover``.

The GPU kernels do the per-pixel work; the bi-level coder is host code in the same
library (the paper runs JBIG-KIT on the host as well).  This module moves buffers.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import rdhei as rd


def candidate_order(hist) -> list[tuple[int, int]]:
    """(b, capacity) for b = 2..8 in the order of Eq. optimal_b for LMR, from the
    library (rdhei_b_candidates)."""
    return rd.b_candidates(hist, rd.LMR)


@dataclass
class LmrEncoded:
    b: int                     # 0 for a bad case
    enc: torch.Tensor          # device I_e with the container in bit 7
    map_bits: torch.Tensor     # device rot(l_b)
    eta_bits: torch.Tensor     # device rot(eta)
    side_nbits: int
    capacity: int              # (b - 1) zeros(b); 0 for a bad case
    tries: int                 # candidates tried


def lmr_encode(imgs: list[torch.Tensor], params: list[rd.Params], threads: int = 0, stream=None) -> list[LmrEncoded]:
    n = len(imgs)
    dev = imgs[0].device
    st = stream or torch.cuda.current_stream(dev)
    shapes = [tuple(x.shape) for x in imgs]
    enc = [torch.empty_like(x) for x in imgs]
    maps = [rd.bitbuf(x.numel(), dev) for x in imgs]
    etas = [rd.bitbuf(x.numel(), dev) for x in imgs]
    info = rd.new_info(n, dev)
    jobs = [rd.make_job(params[i], *shapes[i], src=imgs[i], dst=enc[i], map_bits=maps[i], eta_bits=etas[i],
                        info=info[i], b=0) for i in range(n)]
    rd.Plan(jobs, st).run(rd.OP_LABEL_ENCRYPT, st)
    st.synchronize()
    inf = rd.read_info(info)
    order = [candidate_order(r["hist"]) for r in inf]
    eta_h = [x.cpu().numpy() for x in etas]
    map_h = [x.cpu().numpy() for x in maps]
    cur = [0] * n                                   # index into order[i]
    b_now = [r["b"] for r in inf]
    assert all(order[i][0][0] == b_now[i] for i in range(n))
    done: dict[int, dict] = {}
    todo = list(range(n))
    while todo:
        packed = rd.lmr_side_pack([(eta_h[i], map_h[i], *shapes[i], b_now[i]) for i in todo], threads)
        retry = []
        for i, r in zip(todo, packed):
            if r["status"] == rd.RDHEI_OK:
                done[i] = r
            elif r["status"] == rd.RDHEI_ECAPACITY and cur[i] + 1 < len(order[i]):
                cur[i] += 1
                b_now[i] = order[i][cur[i]][0]
                retry.append(i)
            elif r["status"] == rd.RDHEI_ECAPACITY:
                done[i] = None                      # bad case
            else:
                raise rd.RdheiError(f"rdhei_lmr_side_pack: status {r['status']} on image {i}")
        if retry:
            # rot(l) of the next b; I_e is the same for every b and stays as computed
            scratch = [torch.empty_like(imgs[i]) for i in retry]
            info2 = rd.new_info(len(retry), dev)
            j2 = [rd.make_job(params[i], *shapes[i], src=imgs[i], dst=scratch[k], map_bits=maps[i], eta_bits=etas[i],
                              info=info2[k], b=b_now[i]) for k, i in enumerate(retry)]
            rd.Plan(j2, st).run(rd.OP_LABEL_ENCRYPT, st)
            st.synchronize()
            for i in retry:
                map_h[i] = maps[i].cpu().numpy()
        todo = retry
    good = [i for i in range(n) if done[i] is not None]
    if good:
        info3 = rd.new_info(len(good), dev)
        sides = [rd.as_bitbuf(torch.from_numpy(done[i]["side"]).to(dev), done[i]["side_nbits"]) for i in good]
        j3 = [rd.make_job(params[i], *shapes[i], dst=enc[i], side_bits=sides[k], side_nbits=done[i]["side_nbits"],
                          info=info3[k]) for k, i in enumerate(good)]
        rd.Plan(j3, st).run(rd.OP_LMR_SET_SIDE, st)
        st.synchronize()
    out = []
    for i in range(n):
        r = done[i]
        b = b_now[i] if r is not None else 0
        out.append(LmrEncoded(b=b, enc=enc[i], map_bits=maps[i], eta_bits=etas[i],
                              side_nbits=r["side_nbits"] if r is not None else 0,
                              capacity=order[i][cur[i]][1] if b else 0, tries=cur[i] + 1))
    return out


def lmr_read_side(imgs: list[torch.Tensor], threads: int = 0, stream=None) -> list[dict]:
    """From images carrying a container in bit 7 (I_e or I_e'): b and the device
    rot(l), rot(eta).  status != 0 marks a malformed container."""
    planes = [rd.msb_plane(x, stream) for x in imgs]
    (stream or torch.cuda.current_stream()).synchronize()
    items = [(p.cpu().numpy(), *x.shape) for p, x in zip(planes, imgs)]
    res = rd.lmr_side_unpack(items, threads)
    dev = imgs[0].device if imgs else "cuda"
    out = []
    for r, x in zip(res, imgs):
        n = x.numel()
        out.append({"status": r["status"], "b": r["b"],
                    "map_bits": rd.as_bitbuf(torch.from_numpy(r["map_bits"]).to(dev), n),
                    "eta_bits": rd.as_bitbuf(torch.from_numpy(r["eta_bits"]).to(dev), n)})
    return out
