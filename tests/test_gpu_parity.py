"""GPU parity: every output of the CUDA path (through the C ABI) equals the CPU
oracle byte for byte -- encrypted image, packed maps, label histogram, b, capacity,
marked image, extracted bits, recovered image.  All arithmetic is integer, so the
bar is bit-exact equality."""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_07992_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rd():
    from paper_2302_07992_gb300 import rdhei
    return rdhei


def _params(rd, variant, seed, **kw):
    k = synth.keys(seed)
    common = dict(variant=variant, k1=k["k1"], nonce1=k["nonce1"], k2=k["k2"], nonce2=k["nonce2"], **kw)
    return rd.Params(**common), oracle.Params(**common)


def _np(t, n=None):
    a = t.detach().cpu().numpy()
    return a if n is None else a[:n]


def _pipeline(rd, img_np, variant, seed, frac=1.0, side_frac=0.4, **kw):
    """Run the four calls on the GPU and the oracle; compare at every stage."""
    H, W = img_np.shape
    p, op = _params(rd, variant, seed, **kw)
    img = torch.from_numpy(img_np).cuda()
    nb = (H * W + 7) // 8
    lmr = (variant & 1) == oracle.LMR
    side_n = int(H * W * side_frac) if lmr else 0
    side = synth.random_bits(seed, side_n) if side_n else None
    side_t = torch.from_numpy(side).cuda() if side_n else None

    e = rd.label_encrypt(img, p, side_t, side_n)
    r = oracle.label_encrypt(op, img_np, side, side_n)
    assert e["hist"] == [int(v) for v in r.hist], "label histogram"
    assert e["b"] == r.b and e["capacity"] == r.capacity, "b / capacity"
    assert np.array_equal(_np(e["enc"]), r.enc), "encrypted image"
    assert np.array_equal(_np(e["map_bits"], nb), r.map_bits), "rotated location map"
    if lmr:
        assert np.array_equal(_np(e["eta_bits"], nb), r.eta_bits), "rotated first-MSB map"

    nbits = int(r.capacity * frac)
    pay = synth.payload_bits(seed, nbits)
    lmr_map = e["map_bits"] if lmr else None
    lmr_map_np = r.map_bits if lmr else None
    m = rd.embed(e["enc"], p, r.b, torch.from_numpy(pay).cuda(), nbits, lmr_map)
    mref, kref = oracle.embed(op, r.b, r.enc, pay, nbits, lmr_map_np)
    assert m["embedded"] == kref
    assert np.array_equal(_np(m["marked"]), mref), "marked image"

    x = rd.extract(m["marked"], p, r.b, nbits, lmr_map)
    xref, xk = oracle.extract(op, r.b, mref, nbits, lmr_map_np)
    assert x["extracted"] == xk
    assert np.array_equal(_np(x["bits"], (xk + 7) // 8), xref), "extracted bits"
    # the zero padding of the last word is part of the contract
    assert not _np(x["bits"])[(xk + 7) // 8:].any() or xk % 8 == 0

    lmr_eta = e["eta_bits"] if lmr else None
    rec = rd.decrypt_recover(m["marked"], p, r.b, lmr_map, lmr_eta)
    rref = oracle.decrypt_recover(op, r.b, mref, lmr_map_np, r.eta_bits if lmr else None)
    assert np.array_equal(_np(rec), rref), "recovered image"
    if lmr:
        assert np.array_equal(rref, img_np)
    return r


SHAPES = [(512, 512), (64, 64), (96, 160), (100, 130), (1, 50), (50, 1), (3, 3), (128, 1024), (200, 72),
          (257, 333), (65, 64), (64, 65), (2, 2), (4096 // 8, 96)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("variant", [oracle.EMR, oracle.LMR])
def test_pipeline_shapes(rd, shape, variant):
    H, W = shape
    seed = H * 1000 + W + variant
    img = synth.synth_image(H, W, seed)
    _pipeline(rd, img, variant, seed)


@pytest.mark.parametrize("variant", [oracle.EMR, oracle.LMR])
@pytest.mark.parametrize("kw", [dict(rot_enable=0), dict(rot_lmin=3), dict(rot_lmin=7), dict(b=3), dict(b=5)])
def test_pipeline_parameters(rd, variant, kw):
    img = synth.synth_image(256, 320, 5, noise_sigma=2.0)
    _pipeline(rd, img, variant, 17, **kw)


@pytest.mark.parametrize("frac", [0.0, 0.01, 0.5, 1.0, 1.7])
def test_partial_and_excess_payload(rd, frac):
    img = synth.synth_image(192, 256, 9)
    _pipeline(rd, img, oracle.EMR, 23, frac=frac)


def test_edge_images(rd):
    # constant (every non-first pixel redundant, b = 7) and no redundancy (capacity 0)
    _pipeline(rd, np.full((130, 200), 91, np.uint8), oracle.EMR, 31)
    _pipeline(rd, np.full((130, 200), 91, np.uint8), oracle.LMR, 31)
    stripes = np.tile(np.array([0, 255], np.uint8), (70, 90))
    _pipeline(rd, stripes, oracle.EMR, 32)
    noise = np.random.default_rng(3).integers(0, 256, size=(300, 300)).astype(np.uint8)
    _pipeline(rd, noise, oracle.EMR, 33)


def test_c1_full_size(rd):
    """One 512 x 512 image, EMR, full-capacity payload (the paper's test-image size)."""
    img = synth.synth_image(512, 512, synth.image_seed(1, 0))
    r = _pipeline(rd, img, oracle.EMR, synth.image_seed(1, 0))
    assert r.capacity > 0
