"""Pins for the oracle's keystream, location maps, label histogram and choice of b.

Each check compares the oracle with something other than itself: a library cipher,
a published test vector, the adjacent-pixel definition the paper states, brute force,
or a closed-form special case.
"""
import json
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- keystream --
def test_chacha_block_rfc8439_vector():
    g = json.load(open(os.path.join(GOLD, "rfc8439_block.json")))
    out = oracle.chacha20_block(bytes.fromhex(g["key_hex"]), g["counter"], bytes.fromhex(g["nonce_hex"]))
    assert bytes(out).hex() == g["block_hex"]


@pytest.mark.parametrize("nbytes", [1, 63, 64, 65, 1000, 4096 + 17])
def test_keystream_matches_library_chacha20(nbytes):
    ciphers = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    rng = np.random.default_rng(nbytes)
    key = bytes(rng.integers(0, 256, 32, dtype=np.uint8))
    nonce = bytes(rng.integers(0, 256, 12, dtype=np.uint8))
    # library nonce = 32-bit little-endian block counter (0) followed by the 96-bit nonce
    enc = ciphers.Cipher(ciphers.algorithms.ChaCha20(key, bytes(4) + nonce), mode=None).encryptor()
    ref = np.frombuffer(enc.update(bytes(nbytes)), np.uint8)
    assert np.array_equal(oracle.keystream(key, nonce, nbytes), ref)


# ----------------------------------------------------------- location maps --
def _adjacent_labels(img, b):
    """Label 1 where the top b bits differ from the left neighbour's (column 0 -> 1):
    the paper's own description of the map ("directly compare the MSBs of adjacent
    pixels", Sec. III), an independent statement of the glide rule."""
    m = (img >> (8 - b)).astype(np.int32)
    L = np.ones_like(img)
    L[:, 1:] = (m[:, 1:] != m[:, :-1]).astype(np.uint8)
    return L


def test_glide_all_pixel_pairs_exhaustive():
    a = np.arange(65536, dtype=np.uint32)
    img = np.stack([(a >> 8) & 0xFF, a & 0xFF], axis=1).astype(np.uint8)   # every (left, right) pair
    for b in range(1, 9):
        L = oracle.glide_labels(img, b)
        assert np.all(L[:, 0] == 1)
        diff = (img[:, 0] >> (8 - b)) != (img[:, 1] >> (8 - b))
        assert np.array_equal(L[:, 1], diff.astype(np.uint8)), b


@pytest.mark.parametrize("seed", range(6))
def test_glide_equals_adjacent_definition_random_tiny(seed):
    rng = np.random.default_rng(seed)
    H, W = rng.integers(1, 9, size=2)
    # piecewise-constant rows so that long redundant runs occur
    img = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    img[:, W // 2:] = img[:, W // 2:W // 2 + 1]
    for b in range(1, 9):
        assert np.array_equal(oracle.glide_labels(img, b), _adjacent_labels(img, b))


@pytest.mark.parametrize("shape", [(1, 1), (1, 17), (9, 1), (13, 29), (64, 64)])
def test_label_hist_brute_force(shape):
    rng = np.random.default_rng(shape[0] * 100 + shape[1])
    img = np.clip(rng.normal(128, 6, size=shape).cumsum(axis=1) % 256, 0, 255).astype(np.uint8)
    h = oracle.label_hist(img)
    ref = np.zeros(9, np.int64)
    H, W = shape
    for i in range(H):
        ref[0] += 1                                   # first column: no left neighbour
        for j in range(1, W):
            d = int(img[i, j]) ^ int(img[i, j - 1])
            ref[8 - d.bit_length()] += 1              # leading bits shared with the left pixel
    assert h.sum() == H * W
    assert np.array_equal(h.astype(np.int64), ref)
    zeros = [h[b:].sum() for b in range(1, 9)]
    assert all(zeros[i] >= zeros[i + 1] for i in range(7))


def _brute_b(img, variant):
    best, best_b = -1, None
    for b in (range(2, 8) if variant == oracle.EMR else range(2, 9)):
        zeros = int((_adjacent_labels(img, b) == 0).sum())
        cap = (b if variant == oracle.EMR else b - 1) * zeros
        if cap > best:
            best, best_b = cap, b
    return best_b, best


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("variant", [oracle.EMR, oracle.LMR])
def test_choose_b_brute_force(seed, variant):
    rng = np.random.default_rng(seed)
    H, W = rng.integers(4, 40, size=2)
    sigma = [0.5, 2, 8, 30][seed % 4]
    img = np.clip(128 + rng.normal(0, sigma, size=(H, W)).cumsum(axis=1) * 0.2
                  + rng.normal(0, sigma, size=(H, W)), 0, 255).astype(np.uint8)
    b_ref, cap_ref = _brute_b(img, variant)
    h = oracle.label_hist(img)
    assert oracle.choose_b(variant, h) == b_ref
    enc = oracle.label_encrypt(oracle.Params(variant=variant), img)
    assert enc.b == b_ref and enc.capacity == cap_ref


@pytest.mark.parametrize("W", [1, 2, 7, 512])
def test_constant_image_max_der(W):
    H = 5
    img = np.full((H, W), 77, np.uint8)
    e = oracle.label_encrypt(oracle.Params(variant=oracle.EMR), img)
    if W == 1:
        assert e.capacity == 0 and e.b == 2           # no redundant pixel at all
    else:
        assert e.b == 7
        assert e.capacity == 7 * H * (W - 1)          # DER = 7 (W - 1) / W
    l = oracle.label_encrypt(oracle.Params(variant=oracle.LMR), img)
    if W > 1:
        assert l.b == 8 and l.capacity == 7 * H * (W - 1)


def test_no_redundancy_gives_zero_capacity():
    img = np.tile(np.array([0, 255], np.uint8), (6, 8))  # every neighbour differs in bit 7
    e = oracle.label_encrypt(oracle.Params(), img)
    assert e.b == 2 and e.capacity == 0
