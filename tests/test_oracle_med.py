"""Pins for the oracle's related-work variant: the MED (LOCO-I) predictor that Sec. II
quotes from Puyang et al. and Puteaux et al., used in place of the paper's glide.

References other than the oracle itself: what the median edge detector is known to
predict exactly (edges along one axis, one-directional ramps, planes whose gradients
have opposite signs), nesting of the b-MSB maps, the full encode / hide / extract /
recover cycle (lossless for LMR, LSB-only loss for EMR, exact payload) and the
capacity identity."""
import numpy as np
import pytest

import oracle
from paper_2302_07992_gb300 import synth


def _params(variant, seed, **kw):
    k = synth.keys(seed)
    return oracle.Params(variant=variant, k1=k["k1"], nonce1=k["nonce1"], k2=k["k2"], nonce2=k["nonce2"], **kw)


def _stripes(H, W, seed, vertical):
    """Image that is constant along one axis, with 5 random edges across the other.
    Returns the image and the number of edges."""
    rng = np.random.default_rng(seed)
    n = W if vertical else H
    cuts = np.sort(rng.choice(np.arange(1, n), size=min(5, n - 1), replace=False)) if n > 1 else np.zeros(0, int)
    vals = rng.integers(0, 256, len(cuts) + 1)
    # neighbouring regions get different values
    for k in range(1, len(vals)):
        if vals[k] == vals[k - 1]:
            vals[k] = (vals[k] + 1) % 256
    line = vals[np.searchsorted(cuts, np.arange(n), side="right")].astype(np.uint8)
    img = np.broadcast_to(line[None, :] if vertical else line[:, None], (H, W)).copy()
    return img, len(cuts)


@pytest.mark.parametrize("shape", [(16, 16), (33, 47), (1, 20), (20, 1)])
@pytest.mark.parametrize("vertical", [True, False])
def test_edges_along_one_axis_are_predicted(shape, vertical):
    """MED predicts the pixel right of a vertical edge from above and the pixel below a
    horizontal edge from the left; only pixel (0, 0) and the edge pixels of the border
    row / column (which predict from one side) stay unpredicted."""
    H, W = shape
    img, ncut = _stripes(H, W, H + W, vertical)
    h = oracle.med_hist(img, seven=False)
    border_edges = ncut if (vertical and H >= 1) or (not vertical and W >= 1) else 0
    assert int(h[8]) == img.size - 1 - border_edges
    # the left-neighbour glide misses every vertical-edge pixel of every row
    if vertical and H > 1 and ncut:
        assert int(oracle.label_hist(img)[8]) < int(h[8])


def test_seven_bit_prediction_ignores_the_lsb():
    img, ncut = _stripes(24, 24, 3, vertical=True)
    h = oracle.med_hist(img, seven=True)
    t8 = oracle.med_labels(img, 7, seven=True)
    assert int(t8.sum()) == 1 + ncut                 # (0, 0) and the row-0 edge pixels
    noisy = img ^ np.random.default_rng(4).integers(0, 2, img.shape).astype(np.uint8)
    assert np.array_equal(oracle.med_labels(noisy, 7, seven=True), t8)
    # predictions carry a zero LSB: a predicted pixel matches in 8 bits iff it is even
    pred_ok = t8 == 0
    assert int(h[8]) == int(np.count_nonzero(pred_ok & ((img & 1) == 0)))


def test_ramps_and_planes():
    i, j = np.mgrid[0:40, 0:50]
    # one-directional ramps: exact everywhere but the border that predicts along the ramp
    assert oracle.med_hist((j * 3).astype(np.uint8), seven=False)[8] == 40 * 50 - 50    # row 0 (left) misses
    assert oracle.med_hist((i * 2).astype(np.uint8), seven=False)[8] == 40 * 50 - 40    # column 0 (up) misses
    plane = (100 + i - j).astype(np.uint8)                                  # opposite-sign gradients
    t8 = oracle.med_labels(plane, 8, seven=False)
    assert t8[1:, 1:].sum() == 0                                             # interior: A + B - C is exact
    assert t8[0, 1:].all() and t8[1:, 0].all()                               # borders predict from one side


def test_maps_are_nested_and_match_the_histogram():
    img = synth.synth_image(45, 61, 5, noise_sigma=3.0)
    for seven in (False, True):
        h = oracle.med_hist(img, seven)
        prev = None
        for b in range(1, 9):
            lb = oracle.med_labels(img, b, seven)
            assert int((lb == 0).sum()) == int(h[b:].sum())
            if prev is not None:
                assert np.all(lb >= prev)                 # redundant for b implies redundant for b - 1
            prev = lb
        assert oracle.med_labels(img, 1, seven)[0, 0] == 1


@pytest.mark.parametrize("variant", [oracle.EMR_MED, oracle.LMR_MED])
@pytest.mark.parametrize("shape", [(64, 64), (45, 77), (1, 33), (33, 1), (130, 70)])
def test_med_cycle(variant, shape):
    H, W = shape
    seed = H * 7 + W
    img = synth.synth_image(H, W, seed, noise_sigma=2.0)
    p = _params(variant, seed)
    e = oracle.label_encrypt(p, img)
    h = oracle.med_hist(img, seven=variant == oracle.EMR_MED)
    assert np.array_equal(e.hist, h)
    base = variant & 1
    assert e.b == oracle.choose_b(base, h)
    per = e.b if base == oracle.EMR else e.b - 1
    assert e.capacity == per * int(h[e.b:].sum())
    lm = e.map_bits if base == oracle.LMR else None
    pay = synth.payload_bits(seed, e.capacity)
    marked, k = oracle.embed(p, e.b, e.enc, pay, e.capacity, lm)
    assert k == e.capacity
    bits, kk = oracle.extract(p, e.b, marked, e.capacity, lm)
    assert kk == k and np.array_equal(np.unpackbits(bits)[:k], np.unpackbits(pay)[:k])
    rec = oracle.decrypt_recover(p, e.b, marked, lm, e.eta_bits if base == oracle.LMR else None)
    if base == oracle.LMR:
        assert np.array_equal(rec, img)
    else:
        assert np.array_equal(rec & 0xFE, img & 0xFE)


def test_med_beats_the_glide_on_edges():
    """On an image of vertical stripes the MED labels leave more redundant pixels than
    the left-neighbour glide, so the optimal capacity is larger."""
    img, _ = _stripes(96, 96, 9, vertical=True)
    pg, pm = _params(oracle.LMR, 9), _params(oracle.LMR_MED, 9)
    assert oracle.label_encrypt(pm, img).capacity > oracle.label_encrypt(pg, img).capacity
