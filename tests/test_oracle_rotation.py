"""Pins for the oracle's multi-scale block rotation (Eqs. roration / roration2).

Independent references: numpy.rot90 for single-level cases, direct summation of the
keystream for the angles, and a closed-form per-bit description of the composed
rotation (derived in the design notes) for the multi-level case.
"""
import numpy as np
import pytest

import oracle


def _ks(H, W, seed):
    rng = np.random.default_rng(seed)
    key = bytes(rng.integers(0, 256, 32, dtype=np.uint8))
    nonce = bytes(rng.integers(0, 256, 12, dtype=np.uint8))
    return oracle.keystream(key, nonce, H * W).reshape(H, W)


@pytest.mark.parametrize("seed", range(4))
def test_block_angle_is_keystream_sum_mod4(seed):
    H, W = 24, 40
    s = _ks(H, W, seed)
    for L in (1, 2, 3, 4):
        B = 1 << L
        for C1 in range(H >> L):
            for C2 in range(W >> L):
                ref = int(s[C1 * B:(C1 + 1) * B, C2 * B:(C2 + 1) * B].astype(np.int64).sum()) % 4
                assert oracle.block_angle(s, H, W, L, C1, C2) == ref


@pytest.mark.parametrize("n", [1, 2, 3])
@pytest.mark.parametrize("seed", range(6))
def test_single_level_is_numpy_rot90(n, seed):
    B = 1 << n
    s = _ks(B, B, seed)
    img = np.arange(B * B, dtype=np.uint8).reshape(B, B)
    a = int(s.astype(np.int64).sum()) % 4
    enc, = oracle.rotate([img], s, lmin=n, direction=0)         # only the top level n
    assert np.array_equal(enc, np.rot90(img, a))
    dec, = oracle.rotate([enc], s, lmin=n, direction=1)
    assert np.array_equal(dec, img)


def test_remainder_not_rotated():
    H, W = 4, 7                                                   # n = 2: one 4x4 block + 3 spare columns
    s = _ks(H, W, 11)
    img = np.arange(H * W, dtype=np.uint8).reshape(H, W)
    enc, = oracle.rotate([img], s, lmin=2, direction=0)
    a = int(s[:, :4].astype(np.int64).sum()) % 4
    assert np.array_equal(enc[:, :4], np.rot90(img[:, :4], a))
    assert np.array_equal(enc[:, 4:], img[:, 4:])


def _closed_form_dst(H, W, s, lmin):
    """Destination of every pixel under the composed rotation.  A level-L rotation
    by a quarter-turns moves a pixel inside its block as (u, v) -> (B-1-v, u) per
    quarter-turn, i.e. it acts on every coordinate bit below L separately, and it
    never changes bits >= L, which therefore still name the pixel's block at all
    higher levels.  So bit k of the destination is bit k of the source rotated by
    S_k = sum of the angles of the source's enclosing blocks at levels > k."""
    n = oracle.levels(H, W)
    S = s.astype(np.int64)
    ang = {}
    for L in range(max(lmin, 1), n + 1):
        B = 1 << L
        hb, wb = H >> L, W >> L
        sums = S[:hb * B, :wb * B].reshape(hb, B, wb, B).sum(axis=(1, 3)) % 4
        ang[L] = (sums, hb, wb)
    r, c = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    dr, dc = r.copy(), c.copy()
    for k in range(n):
        tot = np.zeros_like(r)
        for L, (sums, hb, wb) in ang.items():
            if L <= k:
                continue
            br, bc = r >> L, c >> L
            inside = (br < hb) & (bc < wb)
            tot += np.where(inside, sums[np.minimum(br, hb - 1), np.minimum(bc, wb - 1)], 0)
        tot %= 4
        u, v = (r >> k) & 1, (c >> k) & 1
        nu, nv = u.copy(), v.copy()
        for q in range(1, 4):                      # apply q quarter-turns where tot == q
            m = tot == q
            uu, vv = u.copy(), v.copy()
            for _ in range(q):
                uu, vv = 1 - vv, uu
            nu[m], nv[m] = uu[m], vv[m]
        dr = (dr & ~(1 << k)) | (nu << k)
        dc = (dc & ~(1 << k)) | (nv << k)
    return dr, dc


@pytest.mark.parametrize("shape,lmin", [((16, 16), 1), ((24, 40), 1), ((33, 65), 1), ((64, 48), 2),
                                        ((40, 40), 4), ((7, 300), 1), ((128, 128), 3)])
def test_multilevel_matches_closed_form(shape, lmin):
    H, W = shape
    s = _ks(H, W, H * 7 + W)
    img = np.random.default_rng(1).integers(0, 256, size=(H, W)).astype(np.uint8)
    enc, = oracle.rotate([img], s, lmin=lmin, direction=0)
    dr, dc = _closed_form_dst(H, W, s, lmin)
    ref = np.zeros_like(img)
    ref[dr, dc] = img
    assert np.array_equal(enc, ref)


@pytest.mark.parametrize("shape,lmin", [((16, 16), 1), ((31, 77), 1), ((64, 64), 4), ((5, 5), 1)])
def test_round_trip_and_permutation(shape, lmin):
    H, W = shape
    s = _ks(H, W, 5)
    img = np.random.default_rng(2).integers(0, 256, size=(H, W)).astype(np.uint8)
    lab = (img & 1).astype(np.uint8)
    e_img, e_lab = oracle.rotate([img, lab], s, lmin=lmin, direction=0)
    assert np.array_equal(np.sort(e_img, axis=None), np.sort(img, axis=None))
    d_img, d_lab = oracle.rotate([e_img, e_lab], s, lmin=lmin, direction=1)
    assert np.array_equal(d_img, img) and np.array_equal(d_lab, lab)
    # planes rotated together stay aligned
    assert np.array_equal(e_lab, e_img & 1)


def test_levels_rule():
    assert oracle.levels(512, 512) == 9                  # block sizes 2^1..2^9 for 512 x 512
    assert oracle.levels(1, 100) == 0
    assert oracle.levels(300, 4096) == 8
    assert oracle.effective_lmin(oracle.LMR, 0, 512, 512) == 4   # 2^4..2^9 for LMR at 512 x 512
    assert oracle.effective_lmin(oracle.EMR, 0, 512, 512) == 1
    assert oracle.effective_lmin(oracle.LMR, 0, 8, 8) == 3
