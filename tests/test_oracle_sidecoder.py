"""Pins for the oracle's LMR side-information coder and fit loop (Sec. III-B-1).

References other than the coder itself: exact round trips, the information content of
the coded symbols under the adaptive model (an arithmetic coder must land within a few
bits of it), causality of the template, near-zero cost of patterns the template sees,
the C oracle's choice of b, and a whole LMR encode -> hide -> extract -> recover cycle
in which the hider and the receiver see only the first MSB plane.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import sidecoder as sc
from paper_2302_07992_gb300 import synth


def _bm(kind, H, W, seed=0):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:H, 0:W]
    if kind == "zeros":
        return np.zeros((H, W), np.uint8)
    if kind == "ones":
        return np.ones((H, W), np.uint8)
    if kind == "random":
        return rng.integers(0, 2, (H, W)).astype(np.uint8)
    if kind == "sparse":
        return (rng.random((H, W)) < 0.05).astype(np.uint8)
    if kind == "cols":
        return (x & 1).astype(np.uint8)
    if kind == "rows":
        return (y & 1).astype(np.uint8)
    if kind == "checker":
        return ((x + y) & 1).astype(np.uint8)
    if kind == "blobs":
        return (((x // 7) * 3 + (y // 5) * 5) % 4 == 0).astype(np.uint8)
    raise ValueError(kind)


KINDS = ["zeros", "ones", "random", "sparse", "cols", "rows", "checker", "blobs"]


@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (9, 1), (2, 2), (3, 5), (17, 23), (40, 64)])
@pytest.mark.parametrize("kind", KINDS)
def test_round_trip(shape, kind):
    bm = _bm(kind, *shape, seed=shape[0] * 7 + shape[1])
    data = sc.encode_bitmap(bm)
    assert np.array_equal(sc.decode_bitmap(data, *shape), bm)


def _ideal_bits(bm):
    """Information content of the symbols under the adaptive model, in bits."""
    H, W = bm.shape
    c0 = [1] * 1024
    c1 = [1] * 1024
    total = 0.0
    for y in range(H):
        for x in range(W):
            ctx = sc.context(bm, y, x)
            p0 = c0[ctx] / (c0[ctx] + c1[ctx])
            bit = int(bm[y, x])
            total -= math.log2(1 - p0 if bit else p0)
            if bit:
                c1[ctx] += 2
            else:
                c0[ctx] += 2
            if c0[ctx] + c1[ctx] > 8192:
                c0[ctx], c1[ctx] = (c0[ctx] >> 1) | 1, (c1[ctx] >> 1) | 1
    return total


@pytest.mark.parametrize("kind", ["random", "sparse", "blobs", "checker"])
def test_code_length_matches_information_content(kind):
    bm = _bm(kind, 48, 64, seed=3)
    ideal = _ideal_bits(bm)
    nbits = 8 * len(sc.encode_bitmap(bm))
    # arithmetic coding: at most 2 terminating bits + byte padding + integer rounding
    assert ideal - 1e-6 <= nbits <= ideal + 2 + 8 + 1e-3 * ideal


def test_template_is_causal_and_complete():
    rng = np.random.default_rng(5)
    bm = rng.integers(0, 2, (9, 11)).astype(np.uint8)
    for y, x in [(0, 0), (4, 5), (8, 10), (3, 0), (0, 7)]:
        c = sc.context(bm, y, x)
        later = bm.copy()
        later[y, x:] ^= 1
        later[y + 1:] ^= 1
        assert sc.context(later, y, x) == c
    # every template neighbour is a distinct context bit
    seen = 0
    for dy, dx in sc.TEMPLATE:
        one = np.zeros((5, 5), np.uint8)
        one[2 + dy, 2 + dx] = 1
        c = sc.context(one, 2, 2)
        assert c and (c & (c - 1)) == 0 and not (c & seen)
        seen |= c
    assert seen == (1 << sc.CTX_BITS) - 1


@pytest.mark.parametrize("kind", ["zeros", "ones", "cols", "rows", "checker"])
def test_patterns_the_template_sees_cost_almost_nothing(kind):
    bm = _bm(kind, 128, 128)
    assert 8 * len(sc.encode_bitmap(bm)) < 0.01 * bm.size


def test_random_bitmap_does_not_compress():
    bm = _bm("random", 64, 64, seed=9)
    assert 8 * len(sc.encode_bitmap(bm)) > 0.97 * bm.size


def test_container_round_trip():
    eta, lm = _bm("blobs", 30, 40), _bm("sparse", 30, 40, seed=2)
    side = sc.pack_side(eta, lm, 5)
    assert side[0] == 5
    le, ll = int.from_bytes(side[1:5], "big"), int.from_bytes(side[5:9], "big")
    assert len(side) == 9 + le + ll
    b, e2, l2 = sc.unpack_side(side + bytes(17), 30, 40)     # the plane continues after the container
    assert b == 5 and np.array_equal(e2, eta) and np.array_equal(l2, lm)


def test_candidate_order_starts_with_the_c_oracle_choice():
    for seed in range(6):
        img = synth.synth_image(40, 56, seed, noise_sigma=1 + 3 * seed)
        hist = oracle.label_hist(img)
        order = sc.candidate_order(hist)
        assert sorted(order) == list(range(2, 9))
        assert order[0] == oracle.choose_b(oracle.LMR, hist)


def test_fit_moves_to_the_next_map_and_reports_bad_cases():
    H, W = 32, 32
    hist = [0, 0, 10, 20, 30, 40, 50, 60, 70]
    order = sc.candidate_order(hist)
    eta = _bm("zeros", H, W)
    noisy = _bm("random", H, W, seed=1)
    # the best candidate's map is incompressible, the others are flat
    b, side = sc.fit(hist, eta, lambda bb: noisy if bb == order[0] else _bm("zeros", H, W), H, W)
    assert b == order[1] and 8 * len(side) <= H * W
    # nothing fits
    b, side = sc.fit(hist, noisy, lambda bb: noisy, H, W)
    assert b == 0 and side is None


def _params(seed, **kw):
    k = synth.keys(seed)
    return oracle.Params(variant=oracle.LMR, k1=k["k1"], nonce1=k["nonce1"], k2=k["k2"], nonce2=k["nonce2"], **kw)


def test_lmr_end_to_end_with_compressed_side_information():
    """Owner: fit loop, maps into the first MSB plane.  Hider and receiver: only the
    marked image (and their keys); the maps come back out of the MSB plane."""
    H, W, seed = 96, 128, 12
    img = synth.synth_image(H, W, seed, noise_sigma=2.0)
    p = _params(seed)
    first = oracle.label_encrypt(p, img)
    eta = sc.unpack_bits(first.eta_bits, H, W)

    def lmap_of(b):
        return sc.unpack_bits(oracle.label_encrypt(_params(seed, b=b), img).map_bits, H, W)

    b, side = sc.fit(first.hist, eta, lmap_of, H, W)
    assert b >= 2, "synthetic image should be a good case"
    side_bits = np.frombuffer(side, np.uint8)
    e = oracle.label_encrypt(_params(seed, b=b), img, side_bits, 8 * len(side))
    # the hider reads the container from bit 7 of the encrypted image
    plane = np.packbits((e.enc.reshape(-1) >> 7) & 1).tobytes()
    hb, heta, hl = sc.unpack_side(plane, H, W)
    assert hb == b and np.array_equal(hl, sc.unpack_bits(e.map_bits, H, W))
    lmap = np.packbits(hl.reshape(-1))
    pay = synth.payload_bits(seed, e.capacity)
    marked, k = oracle.embed(p, hb, e.enc, pay, e.capacity, lmap)
    assert k == e.capacity > 0
    # the receiver reads the same container from the marked image
    plane2 = np.packbits((marked.reshape(-1) >> 7) & 1).tobytes()
    rb, reta, rl = sc.unpack_side(plane2, H, W)
    bits, kk = oracle.extract(p, rb, marked, e.capacity, np.packbits(rl.reshape(-1)))
    assert kk == e.capacity and np.array_equal(np.unpackbits(bits)[:kk], np.unpackbits(pay)[:kk])
    rec = oracle.decrypt_recover(p, rb, marked, np.packbits(rl.reshape(-1)), np.packbits(reta.reshape(-1)))
    assert np.array_equal(rec, img)
