"""Pins for the oracle's security and quality statistics (Sec. IV-C, Tab. analysis;
PSNR of Sec. III-A; SSIM of Wang et al. 2004, which the paper uses without defining).

References other than the oracle itself: closed forms (uniform and constant
histograms, images that differ by one grey level everywhere, constant image pairs),
scipy's entropy and Pearson chi-square routines, brute-force Python loops on tiny
images, the expectations of two independent uniform images, and the printed table
values in tests/golden/tab_analysis.json.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.stats

import oracle
from oracle import metrics as M
from paper_2302_07992_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _uniform_image(H, W, seed):
    """Every grey level exactly H W / 256 times, in random positions."""
    assert (H * W) % 256 == 0
    v = np.arange(H * W, dtype=np.int64) % 256
    return np.random.default_rng(seed).permutation(v).astype(np.uint8).reshape(H, W)


# ----------------------------------------------------------- one image --
def test_entropy_closed_forms():
    assert abs(M.entropy(_uniform_image(64, 64, 1)) - 8.0) < 1e-12
    assert M.entropy(np.full((9, 7), 77, np.uint8)) == 0.0
    half = np.zeros((8, 8), np.uint8)
    half[:4] = 255
    assert abs(M.entropy(half) - 1.0) < 1e-15
    four = (np.arange(64) % 4 * 60).astype(np.uint8).reshape(8, 8)
    assert abs(M.entropy(four) - 2.0) < 1e-15


def test_entropy_and_chi2_match_scipy():
    img = synth.synth_image(96, 80, 5)
    h = np.bincount(img.ravel(), minlength=256)
    assert abs(M.entropy(img) - scipy.stats.entropy(h, base=2)) < 1e-12
    # the printed formula is Pearson's statistic against equal expected counts N/256
    ref = scipy.stats.chisquare(h).statistic
    assert abs(M.chi2(img) - ref) < 1e-9 * max(1.0, ref)


def test_chi2_closed_forms():
    assert abs(M.chi2(_uniform_image(32, 32, 2))) < 1e-9
    N = 13 * 11
    assert abs(M.chi2(np.full((13, 11), 200, np.uint8)) - 255.0 * N) < 1e-9 * N


def test_histogram_counts():
    img = np.array([[0, 255, 3], [3, 3, 255]], np.uint8)
    h = M.histogram(img)
    assert h.sum() == 6 and h[0] == 1 and h[3] == 3 and h[255] == 2


# ------------------------------------------------------------ image pairs --
def test_pair_closed_forms():
    a = synth.synth_image(40, 56, 7)
    assert M.npcr(a, a) == 0.0 and M.uaci(a, a) == 0.0 and M.psnr(a, a) == math.inf
    b = a ^ 1                                         # every pixel off by exactly one level
    assert M.npcr(a, b) == 100.0
    assert abs(M.uaci(a, b) - 100.0 / 255.0) < 1e-12
    assert abs(M.psnr(a, b) - 20.0 * math.log10(255.0)) < 1e-12
    z, f = np.zeros((5, 6), np.uint8), np.full((5, 6), 255, np.uint8)
    assert M.npcr(z, f) == 100.0 and abs(M.uaci(z, f) - 100.0) < 1e-12 and abs(M.psnr(z, f)) < 1e-12


def test_psnr_half_lsb_flips_is_the_printed_model():
    g = json.load(open(os.path.join(GOLD, "paper_numbers.json")))["emr_expected_psnr_db"]["value"]
    a = synth.synth_image(64, 64, 9)
    b = a.copy()
    b[::2] ^= 1                                       # MSE exactly 1/2
    assert abs(M.psnr(a, b) - g) < 5e-5
    assert abs(M.npcr(a, b) - 50.0) < 1e-12


def test_pair_brute_force_tiny():
    rng = np.random.default_rng(11)
    a = rng.integers(0, 256, (7, 5)).astype(np.uint8)
    b = rng.integers(0, 256, (7, 5)).astype(np.uint8)
    b[2, 3] = a[2, 3]
    n_diff = sum_abs = sum_sq = 0
    for i in range(7):
        for j in range(5):
            d = abs(int(a[i, j]) - int(b[i, j]))
            n_diff += d != 0
            sum_abs += d
            sum_sq += d * d
    s = M.image_stats(a, b)
    assert (s["n_diff"], s["sum_abs"], s["sum_sq"]) == (n_diff, sum_abs, sum_sq)
    assert abs(s["npcr"] - 100.0 * n_diff / 35) < 1e-12
    assert abs(s["uaci"] - 100.0 * sum_abs / (255 * 35)) < 1e-12
    assert abs(s["psnr"] - 10 * math.log10(255 ** 2 * 35 / sum_sq)) < 1e-12


def test_independent_uniform_pair_expectations():
    """Two independent uniform images: NPCR -> 255/256, UACI -> E|X-Y|/255 with
    E|X-Y| = (256^2 - 1) / (3 * 256)."""
    rng = np.random.default_rng(12)
    n = 1 << 20
    a = rng.integers(0, 256, n).astype(np.uint8).reshape(1024, 1024)
    b = rng.integers(0, 256, n).astype(np.uint8).reshape(1024, 1024)
    p = 255.0 / 256.0
    assert abs(M.npcr(a, b) - 100 * p) < 5 * 100 * math.sqrt(p * (1 - p) / n)
    mean_abs = (256 ** 2 - 1) / (3 * 256)
    sd_abs = math.sqrt((256 ** 2 - 1) * (256 ** 2 + 2) / (18 * 256 ** 2))   # sd of |X-Y|
    assert abs(M.uaci(a, b) - 100 * mean_abs / 255) < 5 * 100 * sd_abs / 255 / math.sqrt(n)


# ------------------------------------------------------------------- SSIM --
def test_gaussian_window():
    w = M.gaussian_window()
    assert w.shape == (11, 11)
    assert abs(w.sum() - 1.0) < 1e-14
    assert np.allclose(w, w.T) and np.allclose(w, w[::-1, ::-1])
    g = np.exp(-np.arange(-5, 6) ** 2 / (2 * 1.5 ** 2))
    g /= g.sum()
    assert np.allclose(w, np.outer(g, g), rtol=0, atol=1e-16)
    assert abs(w[5, 5] / w[5, 6] - math.exp(1 / 4.5)) < 1e-12


def test_ssim_identical_and_symmetric():
    a = synth.synth_image(40, 33, 13)
    assert abs(M.ssim(a, a) - 1.0) < 1e-12
    b = synth.synth_image(40, 33, 14)
    assert abs(M.ssim(a, b) - M.ssim(b, a)) < 1e-12
    assert math.isnan(M.ssim(a[:10], b[:10]))


def test_ssim_constant_pair_closed_form():
    for c1, c2 in [(10, 200), (128, 129), (0, 255)]:
        a = np.full((20, 15), c1, np.uint8)
        b = np.full((20, 15), c2, np.uint8)
        want = (2.0 * c1 * c2 + M.SSIM_C1) / (c1 * c1 + c2 * c2 + M.SSIM_C1)
        assert abs(M.ssim(a, b) - want) < 1e-12


def _ssim_one_window(a, b):
    """SSIM of an 11 x 11 image pair: one window, weighted sums by explicit loops."""
    r = 5.0
    w = [[math.exp(-((u - r) ** 2 + (v - r) ** 2) / (2 * 1.5 ** 2)) for v in range(11)] for u in range(11)]
    tot = sum(map(sum, w))
    mu_a = sum(w[u][v] * float(a[u, v]) for u in range(11) for v in range(11)) / tot
    mu_b = sum(w[u][v] * float(b[u, v]) for u in range(11) for v in range(11)) / tot
    va = sum(w[u][v] * (float(a[u, v]) - mu_a) ** 2 for u in range(11) for v in range(11)) / tot
    vb = sum(w[u][v] * (float(b[u, v]) - mu_b) ** 2 for u in range(11) for v in range(11)) / tot
    cv = sum(w[u][v] * (float(a[u, v]) - mu_a) * (float(b[u, v]) - mu_b) for u in range(11) for v in range(11)) / tot
    C1, C2 = (0.01 * 255) ** 2, (0.03 * 255) ** 2
    return (2 * mu_a * mu_b + C1) * (2 * cv + C2) / ((mu_a ** 2 + mu_b ** 2 + C1) * (va + vb + C2))


def test_ssim_brute_force_windows():
    rng = np.random.default_rng(15)
    a = rng.integers(0, 256, (11, 11)).astype(np.uint8)
    b = np.clip(a.astype(int) + rng.integers(-20, 21, (11, 11)), 0, 255).astype(np.uint8)
    assert abs(M.ssim(a, b) - _ssim_one_window(a, b)) < 1e-12
    # 12 x 13: six windows, each checked by the loops
    a = rng.integers(0, 256, (12, 13)).astype(np.uint8)
    b = 255 - a
    m = M.ssim_map(a, b)
    assert m.shape == (2, 3)
    for y in range(2):
        for x in range(3):
            assert abs(m[y, x] - _ssim_one_window(a[y:y + 11, x:x + 11], b[y:y + 11, x:x + 11])) < 1e-12
    assert abs(M.ssim(a, b) - m.mean()) < 1e-15


def test_ssim_independent_noise_near_zero():
    rng = np.random.default_rng(16)
    a = rng.integers(0, 256, (128, 128)).astype(np.uint8)
    b = rng.integers(0, 256, (128, 128)).astype(np.uint8)
    assert abs(M.ssim(a, b)) < 0.02


# ----------------------------------------- the method, against Tab. analysis --
def _keys(seed):
    k = synth.keys(seed)
    return oracle.Params(variant=oracle.LMR, k1=k["k1"], nonce1=k["nonce1"], k2=k["k2"], nonce2=k["nonce2"])


def test_encrypted_image_lands_in_the_printed_band():
    """An LMR encrypted image whose first MSB plane holds random-looking side
    information is uniform whatever the content: its statistics fall where the
    paper's I_e rows are (512 x 512; expected entropy 8 - 255 / (2 N ln 2) = 7.99930,
    expected chi-square 255, i.e. about 16 for the table's root form)."""
    g = json.load(open(os.path.join(GOLD, "tab_analysis.json")))
    rows = g["I_e"].values()
    ent = [v for r in rows for v in r["entropy"]]
    chi_t = [v for r in rows for v in r["chi2_table"]]
    npc = [v for r in rows for v in r["npcr"]]
    H, W = g["size"]
    N = H * W
    for seed in (21, 22):
        img = synth.synth_image(H, W, seed)
        p = _keys(seed)
        e = oracle.label_encrypt(p, img, synth.random_bits(seed, N), N)
        s = M.image_stats(e.enc, img)
        assert min(ent) - 3e-4 <= s["entropy"] <= max(ent) + 3e-4
        assert abs(s["entropy"] - (8 - 255 / (2 * N * math.log(2)))) < 4e-4
        assert min(chi_t) - 4 <= math.sqrt(s["chi2"]) <= max(chi_t) + 4
        assert abs(s["chi2"] - 255) < 5 * math.sqrt(2 * 255)
        assert min(npc) - 0.06 <= s["npcr"] <= max(npc) + 0.06
        assert 5.0 < s["psnr"] < 12.0                      # table: 8.05 .. 9.51 dB
        # the originals are far from uniform, like the table's I rows
        assert s["chi2"] < M.chi2(img) and M.entropy(img) < 7.9


def test_emr_reconstruction_quality():
    """EMR loses only LSBs: PSNR near the printed 51.14 dB model, SSIM close to 1
    (the paper reports 0.9928 for its EMR example)."""
    img = synth.synth_image(256, 256, 23)
    k = synth.keys(23)
    p = oracle.Params(variant=oracle.EMR, k1=k["k1"], nonce1=k["nonce1"], k2=k["k2"], nonce2=k["nonce2"])
    e = oracle.label_encrypt(p, img)
    pay = synth.payload_bits(23, e.capacity)
    marked, _ = oracle.embed(p, e.b, e.enc, pay, e.capacity)
    rec = oracle.decrypt_recover(p, e.b, marked)
    s = M.image_stats(img, rec, with_ssim=True)
    assert abs(s["psnr"] - 51.1411) < 0.1
    assert 49.0 < s["npcr"] < 51.0
    assert 0.97 < s["ssim"] < 1.0
