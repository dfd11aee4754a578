"""GPU parity of rdhei_image_stats against the fp64 oracle statistics.

Exact: the 256-bin histogram, pixels that differ, sum |a - b|, sum (a - b)^2.
fp64 functions of those (entropy, chi-square, NPCR, UACI, PSNR): relative 1e-12.
SSIM: local moments in fp32 with pixels centred at 128; an fp32 emulation of the
same arithmetic stays within 6e-5 of fp64 per window on flat, edge, noise and
synthetic images, so the mean is compared at 1e-4 absolute.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import metrics as M
from paper_2302_07992_gb300 import synth

pytestmark = pytest.mark.gpu

SSIM_TOL = 1e-4


def _rd():
    from paper_2302_07992_gb300 import rdhei
    return rdhei


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def _close(got, want, rel=1e-12):
    if math.isinf(want) or math.isnan(want):
        return got == want or (math.isnan(want) and math.isnan(got))
    return abs(got - want) <= rel * max(1.0, abs(want))


def _check(got, a, b, ssim):
    want = M.image_stats(a, b, with_ssim=ssim)
    assert np.array_equal(np.array(got["hist"]), want["hist"])
    assert _close(got["entropy"], want["entropy"]) and _close(got["chi2"], want["chi2"])
    if b is None:
        assert got["n_diff"] == 0 and got["sum_abs"] == 0 and got["sum_sq"] == 0
        assert math.isnan(got["npcr"]) and math.isnan(got["psnr"]) and math.isnan(got["ssim"])
        return
    assert (got["n_diff"], got["sum_abs"], got["sum_sq"]) == (want["n_diff"], want["sum_abs"], want["sum_sq"])
    assert _close(got["npcr"], want["npcr"]) and _close(got["uaci"], want["uaci"]) and _close(got["psnr"], want["psnr"])
    if ssim and min(a.shape) >= 11:
        assert abs(got["ssim"] - want["ssim"]) < SSIM_TOL, (got["ssim"], want["ssim"])
    else:
        assert math.isnan(got["ssim"])


def _pair(kind, H, W, seed):
    rng = np.random.default_rng(seed)
    a = synth.synth_image(H, W, seed)
    if kind == "random":
        b = rng.integers(0, 256, (H, W)).astype(np.uint8)
    elif kind == "lsb":
        b = a ^ rng.integers(0, 2, (H, W)).astype(np.uint8)
    elif kind == "same":
        b = a.copy()
    elif kind == "other":
        b = synth.synth_image(H, W, seed + 1000)
    else:
        b = None
    return a, b


SHAPES = [(1, 1), (3, 5), (11, 11), (12, 13), (45, 77), (64, 64), (100, 203), (75, 140), (43, 75), (256, 256),
          (1000, 11), (11, 1000), (97, 8193)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kind", ["random", "lsb", "same", "other", "none"])
def test_stats_parity(shape, kind):
    rd = _rd()
    H, W = shape
    a, b = _pair(kind, H, W, H * 131 + W)
    got = rd.image_stats([(_dev(a), None if b is None else _dev(b))], ssim=True)[0]
    _check(got, a, b, ssim=True)


def test_stats_without_ssim_flag():
    rd = _rd()
    a, b = _pair("other", 64, 80, 5)
    got = rd.image_stats([(_dev(a), _dev(b))], ssim=False)[0]
    _check(got, a, b, ssim=False)


def test_constant_images():
    rd = _rd()
    a = np.full((70, 90), 7, np.uint8)
    got = rd.image_stats([(_dev(a), _dev(a))], ssim=True)[0]
    assert got["hist"][7] == 70 * 90 and got["entropy"] == 0.0
    assert abs(got["chi2"] - 255.0 * 70 * 90) < 1e-6
    assert got["psnr"] == math.inf and got["npcr"] == 0.0 and abs(got["ssim"] - 1.0) < SSIM_TOL


def test_batch_of_uneven_pairs_in_one_call():
    """One launch over pairs of different sizes and kinds gives each pair's own result."""
    rd = _rd()
    rng = np.random.default_rng(77)
    pairs, host = [], []
    for i in range(24):
        H, W = int(rng.integers(1, 300)), int(rng.integers(1, 300))
        kind = ["random", "lsb", "same", "other", "none"][i % 5]
        a, b = _pair(kind, H, W, 500 + i)
        host.append((a, b))
        pairs.append((_dev(a), None if b is None else _dev(b)))
    got = rd.image_stats(pairs, ssim=True)
    for g, (a, b) in zip(got, host):
        _check(g, a, b, ssim=True)


def test_encrypted_images_from_the_oracle():
    """Stats of the method's images (made by the oracle): an LMR encrypted image with
    full-plane side bits, and the EMR reconstruction against the original."""
    rd = _rd()
    H = W = 512
    img = synth.synth_image(H, W, 31)
    k = synth.keys(31)
    p_l = oracle.Params(variant=oracle.LMR, k1=k["k1"], nonce1=k["nonce1"], k2=k["k2"], nonce2=k["nonce2"])
    e = oracle.label_encrypt(p_l, img, synth.random_bits(31, H * W), H * W)
    p_e = oracle.Params(variant=oracle.EMR, k1=k["k1"], nonce1=k["nonce1"], k2=k["k2"], nonce2=k["nonce2"])
    ee = oracle.label_encrypt(p_e, img)
    marked, _ = oracle.embed(p_e, ee.b, ee.enc, synth.payload_bits(31, ee.capacity), ee.capacity)
    rec = oracle.decrypt_recover(p_e, ee.b, marked)
    host = [(e.enc, img), (rec, img), (marked, img)]
    got = rd.image_stats([(_dev(x), _dev(y)) for x, y in host], ssim=True)
    for g, (x, y) in zip(got, host):
        _check(g, x, y, ssim=True)
    assert got[0]["entropy"] > 7.999 and abs(got[1]["psnr"] - 51.14) < 0.1


def test_misaligned_and_invalid_jobs():
    rd = _rd()
    base = torch.zeros(64 * 64 + 3, dtype=torch.uint8, device="cuda")
    a = base[1:1 + 48 * 64].view(48, 64)                  # odd address: byte staging path
    b = base[3:3 + 48 * 64].view(48, 64)
    a.copy_(_dev(synth.synth_image(48, 64, 3)))
    b.copy_(_dev(synth.synth_image(48, 64, 4)))
    got = rd.image_stats([(a, b)], ssim=True)[0]
    _check(got, a.cpu().numpy(), b.cpu().numpy(), ssim=True)
    out = rd.new_stats(1)
    j = rd.stats_job(a, b, out[0], True)
    j.flags = 6
    with pytest.raises(rd.RdheiError):
        rd.StatsCall([j])
    j = rd.stats_job(a, b, out[0], True)
    j.H = 0
    with pytest.raises(rd.RdheiError):
        rd.StatsCall([j])


@pytest.mark.slow
def test_full_batch_sampled():
    """The 1000-image 512 x 512 batch in one call; sampled images against the oracle."""
    rd = _rd()
    imgs = [synth.batch_image(9000, i) for i in range(1000)]
    dev = [_dev(x) for x in imgs]
    noisy = [x ^ 1 for x in dev]
    got = rd.image_stats(list(zip(dev, noisy)), ssim=True)
    for i in (0, 1, 499, 998, 999):
        _check(got[i], imgs[i], imgs[i] ^ 1, ssim=True)


def test_one_shot_call_plan_reruns_and_graph():
    """rdhei_image_stats, a plan run twice, and the plan replayed from a CUDA graph
    all give the oracle's answer (the accumulators are cleared inside each run)."""
    rd = _rd()
    host = [_pair("lsb", 70, 129, 41), _pair("other", 200, 64, 42), _pair("none", 33, 17, 43)]
    dev = [(_dev(a), None if b is None else _dev(b)) for a, b in host]
    out = rd.new_stats(3)
    jobs = [rd.stats_job(a, b, out[i], True) for i, (a, b) in enumerate(dev)]
    rd.image_stats_once(jobs)
    for g, (a, b) in zip(rd.read_stats(out), host):
        _check(g, a, b, ssim=True)
    call = rd.StatsCall(jobs)
    out.zero_()
    call.run()
    call.run()
    for g, (a, b) in zip(rd.read_stats(out), host):
        _check(g, a, b, ssim=True)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        call.run(side)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        call.run(torch.cuda.current_stream())
    out.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for g, (a, b) in zip(rd.read_stats(out), host):
        _check(g, a, b, ssim=True)
