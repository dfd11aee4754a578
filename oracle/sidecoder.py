"""Lossless bi-level coder for the LMR side information and the LMR fit loop
(Sec. III-B-1, "Maps generation, rotation, and compression" and "Maps embedding").

TEST INFRASTRUCTURE ONLY: used by ``tests/`` to check the library's host coder; the
product package never imports it.  Plain Python loops, for small images.

The paper compresses the rotated first-MSB map rot(eta) and the rotated location map
rot(l) with the JBIG-KIT library, concatenates the two streams into the first MSB
plane of the encrypted image, and, when they do not fit into H W bits, moves to the
"next most optimal" location map.  JBIG-KIT is not available, so the coder is a
JBIG-style one of this project's design (the paper fixes only "lossless bi-level
compression"):

  * context: 10 causal neighbours of pixel (y, x) -- three of row y-2 (x-1, x, x+1),
    five of row y-1 (x-2 .. x+2), two of row y (x-2, x-1) -- packed into a 10-bit
    number, neighbour order as listed, first one the most significant bit; pixels
    outside the bitmap count as 0;
  * model: per context two counts c0, c1, both starting at 1 and raised by 2 for each
    coded symbol (the Krichevsky-Trofimov estimate); when c0 + c1 exceeds 8192 both
    become (c >> 1) | 1;
  * coder: the binary arithmetic coder of Witten, Neal and Cleary (1987) with 32-bit
    low/high, the interval for symbol 0 being the lower floor(range c0 / (c0 + c1))
    values, pending-bit ("follow") scaling, and two terminating bits; the bit string
    is packed MSB-first and padded with zeros to whole bytes.

Side-information container (bit 7 of pixels 0 .. side_nbits-1, raster order of the
rotated image, MSB-first):
  byte 0       b (2..8)
  bytes 1..4   length of the rot(eta) stream in bytes, big-endian
  bytes 5..8   length of the rot(l) stream in bytes, big-endian
  then the rot(eta) stream, then the rot(l) stream.

Fit loop: the candidate b are 2..8 in decreasing order of (b - 1) zeros(b), ties to
the smaller b (the order of Eq. optimal_b); the first b whose container fits into
H W bits is taken.  If none fits the image is a "bad case" (Tab. LMR_block_size).
"""
from __future__ import annotations

import numpy as np

CTX_BITS = 10
COUNT_LIMIT = 8192
TOP = 1 << 32
HALF = 1 << 31
QUARTER = 1 << 30
HEADER_BYTES = 9

# (dy, dx) of the template, most significant context bit first
TEMPLATE = ((-2, -1), (-2, 0), (-2, 1),
            (-1, -2), (-1, -1), (-1, 0), (-1, 1), (-1, 2),
            (0, -2), (0, -1))


def context(bm: np.ndarray, y: int, x: int) -> int:
    H, W = bm.shape
    c = 0
    for dy, dx in TEMPLATE:
        yy, xx = y + dy, x + dx
        v = int(bm[yy, xx]) if 0 <= yy < H and 0 <= xx < W else 0
        c = (c << 1) | v
    return c


class _Model:
    def __init__(self):
        self.c0 = [1] * (1 << CTX_BITS)
        self.c1 = [1] * (1 << CTX_BITS)

    def counts(self, ctx):
        return self.c0[ctx], self.c1[ctx]

    def update(self, ctx, bit):
        if bit:
            self.c1[ctx] += 2
        else:
            self.c0[ctx] += 2
        if self.c0[ctx] + self.c1[ctx] > COUNT_LIMIT:
            self.c0[ctx] = (self.c0[ctx] >> 1) | 1
            self.c1[ctx] = (self.c1[ctx] >> 1) | 1


def encode_bitmap(bm: np.ndarray) -> bytes:
    """Compress an H x W array of 0/1 values."""
    bm = np.asarray(bm, dtype=np.uint8)
    H, W = bm.shape
    model = _Model()
    low, high, pending = 0, TOP - 1, 0
    out = []

    def emit(bit):
        nonlocal pending
        out.append(bit)
        out.extend([1 - bit] * pending)
        pending = 0

    for y in range(H):
        for x in range(W):
            ctx = context(bm, y, x)
            bit = int(bm[y, x])
            c0, c1 = model.counts(ctx)
            rng = high - low + 1
            split = low + rng * c0 // (c0 + c1) - 1
            if bit:
                low = split + 1
            else:
                high = split
            while True:
                if high < HALF:
                    emit(0)
                elif low >= HALF:
                    emit(1)
                    low -= HALF
                    high -= HALF
                elif low >= QUARTER and high < HALF + QUARTER:
                    pending += 1
                    low -= QUARTER
                    high -= QUARTER
                else:
                    break
                low = 2 * low
                high = 2 * high + 1
            model.update(ctx, bit)
    pending += 1
    emit(0 if low < QUARTER else 1)
    while len(out) % 8:
        out.append(0)
    return bytes(np.packbits(np.array(out, dtype=np.uint8)).tolist()) if out else b""


def decode_bitmap(data: bytes, H: int, W: int) -> np.ndarray:
    """Inverse of encode_bitmap; bits past the end of data read as 0."""
    bits = np.unpackbits(np.frombuffer(bytes(data), dtype=np.uint8)) if len(data) else np.zeros(0, np.uint8)
    pos = 0

    def next_bit():
        nonlocal pos
        v = int(bits[pos]) if pos < len(bits) else 0
        pos += 1
        return v

    bm = np.zeros((H, W), dtype=np.uint8)
    model = _Model()
    low, high = 0, TOP - 1
    value = 0
    for _ in range(32):
        value = (value << 1) | next_bit()
    for y in range(H):
        for x in range(W):
            ctx = context(bm, y, x)
            c0, c1 = model.counts(ctx)
            rng = high - low + 1
            split = low + rng * c0 // (c0 + c1) - 1
            if value <= split:
                bit = 0
                high = split
            else:
                bit = 1
                low = split + 1
            while True:
                if high < HALF:
                    pass
                elif low >= HALF:
                    low -= HALF
                    high -= HALF
                    value -= HALF
                elif low >= QUARTER and high < HALF + QUARTER:
                    low -= QUARTER
                    high -= QUARTER
                    value -= QUARTER
                else:
                    break
                low = 2 * low
                high = 2 * high + 1
                value = 2 * value + next_bit()
            bm[y, x] = bit
            model.update(ctx, bit)
    return bm


def unpack_bits(packed, H: int, W: int) -> np.ndarray:
    """MSB-first packed H W bits -> H x W array of 0/1."""
    return np.unpackbits(np.asarray(packed, dtype=np.uint8))[: H * W].reshape(H, W)


def pack_side(eta: np.ndarray, lmap: np.ndarray, b: int) -> bytes:
    """Container of the two compressed maps (bit arrays H x W)."""
    se, sl = encode_bitmap(eta), encode_bitmap(lmap)
    return bytes([b]) + len(se).to_bytes(4, "big") + len(sl).to_bytes(4, "big") + se + sl


def unpack_side(plane: bytes, H: int, W: int):
    """Container (at the start of the first-MSB plane) -> (b, rot(eta), rot(l))."""
    plane = bytes(plane)
    b = plane[0]
    le = int.from_bytes(plane[1:5], "big")
    ll = int.from_bytes(plane[5:9], "big")
    se = plane[HEADER_BYTES:HEADER_BYTES + le]
    sl = plane[HEADER_BYTES + le:HEADER_BYTES + le + ll]
    return b, decode_bitmap(se, H, W), decode_bitmap(sl, H, W)


def candidate_order(hist) -> list[int]:
    """LMR candidates b = 2..8 by decreasing (b - 1) zeros(b), ties to the smaller b;
    zeros(b) = pixels whose label t is at least b (Eq. optimal_b)."""
    hist = [int(h) for h in hist]
    zeros = {b: sum(hist[b:9]) for b in range(2, 9)}
    return sorted(range(2, 9), key=lambda b: (-(b - 1) * zeros[b], b))


def fit(hist, eta: np.ndarray, lmap_of, H: int, W: int):
    """The fit loop: lmap_of(b) gives rot(l_b) as an H x W bit array.  Returns
    (b, container bytes) for the first candidate that fits into H W bits, else
    (0, None)."""
    for b in candidate_order(hist):
        side = pack_side(eta, lmap_of(b), b)
        if 8 * len(side) <= H * W:
            return b, side
    return 0, None
