"""Pins for the oracle's encryption, data hiding, extraction and recovery.

References other than the oracle itself: the library-pinned keystream, numpy.cumsum
bit offsets, the invariants the paper states (error-free extraction, EMR loss limited
to the LSB plane with PSNR ~ 51.1411 dB, lossless LMR, separability) and the printed
numbers in tests/golden/paper_numbers.json.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2302_07992_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _params(variant, seed, **kw):
    k = synth.keys(seed)
    return oracle.Params(variant=variant, k1=k["k1"], nonce1=k["nonce1"], k2=k["k2"], nonce2=k["nonce2"], **kw)


def _bits(packed, n):
    return np.unpackbits(np.asarray(packed, np.uint8))[:n]


def _img(H, W, seed, sigma=4.0):
    return synth.synth_image(H, W, seed, noise_sigma=sigma)


# ------------------------------------------------------------- encryption --
@pytest.mark.parametrize("variant", [oracle.EMR, oracle.LMR])
def test_encryption_without_rotation(variant):
    H, W = 37, 53
    img = _img(H, W, 3)
    p = _params(variant, 3, rot_enable=0)
    e = oracle.label_encrypt(p, img)
    s = oracle.keystream(p.k1, p.nonce1, H * W).reshape(H, W)
    L = oracle.glide_labels(img, e.b)
    dec = e.enc ^ s
    if variant == oracle.EMR:
        assert np.array_equal(dec & 0xFE, img & 0xFE)              # Eq. image_encryption
        assert np.array_equal(e.enc & 1, L)                         # map in the LSB plane
    else:
        assert np.array_equal(dec, img)
    assert np.array_equal(_bits(e.map_bits, H * W), L.reshape(-1))
    assert np.array_equal(_bits(e.eta_bits, H * W), (img >> 7).reshape(-1))   # Eq. MSB_map


def test_lmr_side_bits_fill_first_msb_plane():
    H, W = 16, 24
    img = _img(H, W, 4)
    p = _params(oracle.LMR, 4)
    side = synth.random_bits(4, 300)
    plain = oracle.label_encrypt(p, img)
    withs = oracle.label_encrypt(p, img, side, 300)
    sb = _bits(side, 300)
    flat_p, flat_s = plain.enc.reshape(-1), withs.enc.reshape(-1)
    assert np.array_equal(flat_s[:300] >> 7, sb)
    assert np.array_equal(flat_s[:300] & 0x7F, flat_p[:300] & 0x7F)
    assert np.array_equal(flat_s[300:], flat_p[300:])
    assert np.array_equal(oracle.lmr_set_side(plain.enc, side, 300), withs.enc)


# ---------------------------------------------------------- hide / extract --
@pytest.mark.parametrize("variant", [oracle.EMR, oracle.LMR])
@pytest.mark.parametrize("frac", [0.0, 0.3, 1.0, 1.5])
def test_embed_extract_roundtrip_and_offsets(variant, frac):
    H, W = 48, 70
    seed = 10 + int(frac * 10)
    img = _img(H, W, seed)
    p = _params(variant, seed)
    e = oracle.label_encrypt(p, img)
    cap = e.capacity
    nbits = int(cap * frac) + (1 if frac == 0.3 else 0)
    pay = synth.payload_bits(seed, nbits)
    lmr_map = e.map_bits if variant == oracle.LMR else None
    marked, k = oracle.embed(p, e.b, e.enc, pay, nbits, lmr_map)
    assert k == min(nbits, cap)
    got, kk = oracle.extract(p, e.b, marked, nbits, lmr_map)
    assert kk == k
    assert np.array_equal(_bits(got, k), _bits(pay, k))             # error-free extraction

    # independent placement check: slot offsets from numpy.cumsum of per-pixel capacity
    labels = (e.enc.reshape(-1) & 1) if variant == oracle.EMR else _bits(e.map_bits, H * W)
    per = np.where(labels == 0, e.b if variant == oracle.EMR else e.b - 1, 0)
    assert per.sum() == cap                                          # capacity = sum of slots
    off = np.concatenate([[0], np.cumsum(per)[:-1]])
    z2 = _bits(oracle.keystream(p.k2, p.nonce2, (max(k, 1) + 7) // 8), max(k, 1))
    ebits = _bits(pay, k) ^ z2[:k]
    top = 7 if variant == oracle.EMR else 6
    flat = marked.reshape(-1)
    for q in np.nonzero(per)[0][:400]:
        for u in range(per[q]):
            kb = off[q] + u
            if kb < k:
                assert (flat[q] >> (top - u)) & 1 == ebits[kb]
    # untouched bits: everything outside the slots equals the encrypted image
    mask = np.zeros(H * W, np.uint8)
    for q in np.nonzero(per)[0]:
        for u in range(per[q]):
            if off[q] + u < k:
                mask[q] |= 1 << (top - u)
    assert np.array_equal(flat & ~mask, e.enc.reshape(-1) & ~mask)


def test_extract_respects_max_bits():
    img = _img(32, 32, 21)
    p = _params(oracle.EMR, 21)
    e = oracle.label_encrypt(p, img)
    pay = synth.payload_bits(21, e.capacity)
    marked, _ = oracle.embed(p, e.b, e.enc, pay, e.capacity)
    got, k = oracle.extract(p, e.b, marked, 100)
    assert k == 100 and np.array_equal(_bits(got, 100), _bits(pay, 100))
    got, k = oracle.extract(p, e.b, marked, e.capacity + 999)
    assert k == e.capacity


# --------------------------------------------------------------- recovery --
@pytest.mark.parametrize("shape", [(64, 64), (45, 77), (1, 50), (50, 1), (3, 3)])
def test_emr_recovery_only_lsb_lost(shape):
    H, W = shape
    img = _img(H, W, 31)
    p = _params(oracle.EMR, 31)
    e = oracle.label_encrypt(p, img)
    pay = synth.payload_bits(31, e.capacity)
    marked, _ = oracle.embed(p, e.b, e.enc, pay, e.capacity)
    rec = oracle.decrypt_recover(p, e.b, marked)
    assert np.array_equal(rec & 0xFE, img & 0xFE)


def test_emr_psnr_at_512_matches_paper_model():
    g = json.load(open(os.path.join(GOLD, "paper_numbers.json")))
    img = _img(512, 512, 41)
    p = _params(oracle.EMR, 41)
    e = oracle.label_encrypt(p, img)
    pay = synth.payload_bits(41, e.capacity)
    marked, _ = oracle.embed(p, e.b, e.enc, pay, e.capacity)
    rec = oracle.decrypt_recover(p, e.b, marked)
    mse = np.mean((rec.astype(np.float64) - img) ** 2)
    psnr = 10 * math.log10(255 ** 2 / mse)
    model = g["emr_expected_psnr_db"]["value"]
    assert abs(10 * math.log10(255 ** 2 / 0.5) - model) < 5e-5
    assert abs(psnr - model) < 0.05          # Binomial(262144, 1/2) LSB flips: sigma ~ 0.009 dB


@pytest.mark.parametrize("shape,seed", [((64, 64), 1), ((45, 77), 2), ((512, 512), 3), ((1, 9), 4), ((17, 1), 5)])
def test_lmr_lossless(shape, seed):
    H, W = shape
    img = _img(H, W, 50 + seed, sigma=2.0)
    p = _params(oracle.LMR, 50 + seed)
    e = oracle.label_encrypt(p, img)
    side_n = (H * W) // 3
    side = synth.random_bits(seed, side_n)
    enc = oracle.lmr_set_side(e.enc, side, side_n)
    pay = synth.payload_bits(seed, e.capacity)
    marked, k = oracle.embed(p, e.b, enc, pay, e.capacity, e.map_bits)
    assert k == e.capacity
    assert np.array_equal(marked.reshape(-1)[:side_n] >> 7, _bits(side, side_n))   # side plane intact
    rec = oracle.decrypt_recover(p, e.b, marked, e.map_bits, e.eta_bits)
    assert np.array_equal(rec, img)


def test_separability():
    img = _img(40, 56, 61)
    p = _params(oracle.EMR, 61)
    e = oracle.label_encrypt(p, img)
    pay = synth.payload_bits(61, e.capacity)
    marked, _ = oracle.embed(p, e.b, e.enc, pay, e.capacity)
    wrong = _params(oracle.EMR, 62)
    only_k2 = oracle.Params(variant=oracle.EMR, k1=wrong.k1, nonce1=wrong.nonce1, k2=p.k2, nonce2=p.nonce2)
    only_k1 = oracle.Params(variant=oracle.EMR, k1=p.k1, nonce1=p.nonce1, k2=wrong.k2, nonce2=wrong.nonce2)
    got, _ = oracle.extract(only_k2, e.b, marked, e.capacity)
    assert np.array_equal(_bits(got, e.capacity), _bits(pay, e.capacity))
    rec = oracle.decrypt_recover(only_k1, e.b, marked)
    assert np.array_equal(rec & 0xFE, img & 0xFE)


# ------------------------------------------------------- printed numbers --
def test_lmr_slots_per_redundant_pixel_match_printed_ders():
    """LMR gives b-1 of the b replaced bits to the payload (Sec. III-B-2); the printed
    maximum DERs of both methods on the same images obey LMR = EMR (b-1)/b for b = 4
    (Lena, stated) and b = 5 (Airplane, Crowd)."""
    g = json.load(open(os.path.join(GOLD, "paper_numbers.json")))
    assert g["lena_emr"]["b"] == g["lena_lmr"]["b"] == 4
    for name, b in (("Lena", 4), ("Airplane", 5), ("Crowd", 5)):
        emr, lmr = g["max_der_emr_lmr"][name]
        assert round(emr * (b - 1) / b, 4) == pytest.approx(lmr, abs=1e-4)
    # and the oracle's capacities obey the same ratio on a synthetic image at equal b
    img = _img(128, 128, 71)
    for b in (3, 4, 5):
        ce = oracle.label_encrypt(oracle.Params(variant=oracle.EMR, b=b), img).capacity
        cl = oracle.label_encrypt(oracle.Params(variant=oracle.LMR, b=b), img).capacity
        assert cl * b == ce * (b - 1)


def test_lena_psnr_consistent_with_lsb_model():
    g = json.load(open(os.path.join(GOLD, "paper_numbers.json")))
    mse = 255 ** 2 / 10 ** (g["lena_emr"]["psnr_db"] / 10)
    assert abs(mse - 0.5) < 0.002            # ~half of the LSBs flipped, nothing else lost
