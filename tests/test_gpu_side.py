"""LMR end to end with the side information in the first MSB plane, on the GPU, against
the oracle: the fit loop's b and container, I_e, the maps the hider and receiver read
back from the plane, the marked image, the extracted bits and the lossless recovery."""
import numpy as np
import pytest
import torch

import oracle
from oracle import sidecoder as sc
from paper_2302_07992_gb300 import synth

pytestmark = pytest.mark.gpu


def _mods():
    from paper_2302_07992_gb300 import rdhei, side
    return rdhei, side


def _params(rd, seed, b=0):
    k = synth.keys(seed)
    return rd.Params(variant=rd.LMR, k1=k["k1"], nonce1=k["nonce1"], k2=k["k2"], nonce2=k["nonce2"], b=b)


def _oparams(seed, b=0):
    k = synth.keys(seed)
    return oracle.Params(variant=oracle.LMR, k1=k["k1"], nonce1=k["nonce1"], k2=k["k2"], nonce2=k["nonce2"], b=b)


def _oracle_owner(img, seed):
    H, W = img.shape
    first = oracle.label_encrypt(_oparams(seed), img)
    eta = sc.unpack_bits(first.eta_bits, H, W)
    b, side = sc.fit(first.hist, eta,
                     lambda bb: sc.unpack_bits(oracle.label_encrypt(_oparams(seed, bb), img).map_bits, H, W), H, W)
    if not b:
        return 0, None, None
    e = oracle.label_encrypt(_oparams(seed, b), img, np.frombuffer(side, np.uint8), 8 * len(side))
    return b, side, e


def test_msb_plane():
    rd, _ = _mods()
    rng = np.random.default_rng(3)
    for H, W in [(1, 1), (7, 9), (33, 64), (100, 301)]:
        img = rng.integers(0, 256, (H, W)).astype(np.uint8)
        got = rd.msb_plane(torch.from_numpy(img).cuda()).cpu().numpy()
        want = np.packbits((img.reshape(-1) >> 7) & 1)
        assert np.array_equal(got[: want.size], want)


SHAPES = [(64, 64), (96, 128), (77, 150), (130, 97), (256, 256)]


def test_lmr_cycle_with_side_information():
    rd, side = _mods()
    imgs = [synth.synth_image(H, W, 40 + i, noise_sigma=1.5 + i) for i, (H, W) in enumerate(SHAPES)]
    seeds = [40 + i for i in range(len(SHAPES))]
    dev = [torch.from_numpy(x).cuda() for x in imgs]
    res = side.lmr_encode(dev, [_params(rd, s) for s in seeds], threads=4)
    for i, (img, s, r) in enumerate(zip(imgs, seeds, res)):
        H, W = img.shape
        b, cont, e = _oracle_owner(img, s)
        assert r.b == b, i
        if not b:
            continue
        assert np.array_equal(r.enc.cpu().numpy(), e.enc), i
        assert r.side_nbits == 8 * len(cont)
        # hider: the maps come back out of I_e's MSB plane
        got = side.lmr_read_side([r.enc])[0]
        assert got["status"] == 0 and got["b"] == b
        n = (H * W + 7) // 8
        assert np.array_equal(got["map_bits"].cpu().numpy()[:n], e.map_bits)
        assert np.array_equal(got["eta_bits"].cpu().numpy()[:n], e.eta_bits)
        pay = synth.payload_bits(s, e.capacity)
        p = _params(rd, s)
        marked = rd.embed(r.enc, p, got["b"], torch.from_numpy(pay).cuda(), e.capacity, lmr_map=got["map_bits"])
        mref, _ = oracle.embed(_oparams(s), b, e.enc, pay, e.capacity, e.map_bits)
        marked_t = marked["marked"] if isinstance(marked, dict) else marked
        assert np.array_equal(marked_t.cpu().numpy(), mref), i
        # receiver: reads the same container from the marked image
        rr = side.lmr_read_side([marked_t])[0]
        assert rr["b"] == b
        ex = rd.extract(marked_t, p, rr["b"], e.capacity, lmr_map=rr["map_bits"])
        bits = ex["bits"] if isinstance(ex, dict) else ex
        kk = e.capacity
        assert np.array_equal(np.unpackbits(bits.cpu().numpy())[:kk], np.unpackbits(pay)[:kk]), i
        rec = rd.decrypt_recover(marked_t, p, rr["b"], lmr_map=rr["map_bits"], lmr_eta=rr["eta_bits"])
        rec_t = rec["recovered"] if isinstance(rec, dict) else rec
        assert np.array_equal(rec_t.cpu().numpy(), img), i


def test_fit_loop_moves_past_a_map_that_does_not_fit():
    """A noisy image whose best map is too complex: the library takes the same later b
    as the oracle (or reports the same bad case)."""
    rd, side = _mods()
    rng = np.random.default_rng(8)
    H, W = 64, 64
    base = synth.synth_image(H, W, 8, noise_sigma=1.0).astype(np.int64)
    img = np.clip(base + rng.integers(-40, 41, (H, W)) * (rng.random((H, W)) < 0.5), 0, 255).astype(np.uint8)
    r = side.lmr_encode([torch.from_numpy(img).cuda()], [_params(rd, 8)])[0]
    b, cont, e = _oracle_owner(img, 8)
    assert r.b == b
    if b:
        assert np.array_equal(r.enc.cpu().numpy(), e.enc)
