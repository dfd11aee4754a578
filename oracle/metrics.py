"""Security and quality statistics of the paper's Sec. IV-C (Tab. analysis) and Sec. IV
(PSNR / SSIM of reconstructed images), written out in fp64 numpy.

TEST INFRASTRUCTURE ONLY: used by ``tests/`` to check the device statistics; the
product package never imports it.

Readings taken where the paper is silent or garbled:
  * NPCR counts the pixels that DIFFER between the two images.  The printed indicator
    is 1 where the pixels are equal, but the table values (about 99.6 % between an
    image and its encryption) only fit the "differ" form.
  * 0 * log2(0) = 0 in the entropy sum.
  * PSNR of two equal images is +inf (the paper writes PSNR -> +inf for LMR).
  * SSIM is not defined in the paper; it is Wang et al. 2004 ("Image quality
    assessment: from error visibility to structural similarity"): an 11 x 11
    Gaussian window with sigma 1.5 normalised to sum 1, C1 = (0.01 L)^2,
    C2 = (0.03 L)^2 with L = 255, local statistics taken at every window position
    fully inside the image, the mean over those positions reported.  Images smaller
    than the window give NaN.
"""
from __future__ import annotations

import math

import numpy as np

SSIM_WIN = 11
SSIM_SIGMA = 1.5
SSIM_L = 255.0
SSIM_C1 = (0.01 * SSIM_L) ** 2
SSIM_C2 = (0.03 * SSIM_L) ** 2


def histogram(a: np.ndarray) -> np.ndarray:
    """Grey-level counts of an 8-bit image (256 bins)."""
    return np.bincount(np.asarray(a, dtype=np.uint8).ravel(), minlength=256).astype(np.int64)


def entropy(a: np.ndarray) -> float:
    """Sec. IV-C, Shannon entropy: H(I) = -sum_i P(alpha_i) log2 P(alpha_i)."""
    h = histogram(a)
    n = float(h.sum())
    total = 0.0
    for count in h:
        if count:
            p = count / n
            total -= p * math.log2(p)
    return total


def chi2(a: np.ndarray) -> float:
    """Sec. IV-C, chi-square test: 256 (h w) sum_i (P(alpha_i) - 1/256)^2."""
    h = histogram(a)
    n = float(h.sum())
    s = 0.0
    for count in h:
        d = count / n - 1.0 / 256.0
        s += d * d
    return 256.0 * n * s


def npcr(a: np.ndarray, b: np.ndarray) -> float:
    """Sec. IV-C, NPCR: percentage of pixel positions where the two images differ."""
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    assert a.shape == b.shape
    return float(np.count_nonzero(a != b)) / a.size * 100.0


def uaci(a: np.ndarray, b: np.ndarray) -> float:
    """Sec. IV-C, UACI: mean of |I - I'| / 255, in percent."""
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    assert a.shape == b.shape
    return float(np.abs(a - b).sum()) / (255.0 * a.size) * 100.0


def mse(a: np.ndarray, b: np.ndarray) -> float:
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    return float(((a - b) ** 2).sum()) / a.size


def psnr(a: np.ndarray, b: np.ndarray) -> float:
    """PSNR = 10 log10(255^2 / MSE) (Sec. III-A, Sec. IV); +inf for equal images."""
    m = mse(a, b)
    return math.inf if m == 0.0 else 10.0 * math.log10(255.0 * 255.0 / m)


def gaussian_window(size: int = SSIM_WIN, sigma: float = SSIM_SIGMA) -> np.ndarray:
    """w(u, v) proportional to exp(-(u^2 + v^2) / (2 sigma^2)) on a size x size grid
    centred on 0, normalised so that the weights sum to 1."""
    r = (size - 1) / 2.0
    u = np.arange(size, dtype=np.float64) - r
    w = np.exp(-(u[:, None] ** 2 + u[None, :] ** 2) / (2.0 * sigma * sigma))
    return w / w.sum()


def ssim_map(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Per-window SSIM (Wang et al. 2004, Eq. 13 with the Gaussian-weighted local
    statistics of their Eqs. 14-16) at every window position inside the image."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    assert a.shape == b.shape
    H, W = a.shape
    k = SSIM_WIN
    if H < k or W < k:
        return np.zeros((0, 0))
    w = gaussian_window()
    wa = np.lib.stride_tricks.sliding_window_view(a, (k, k))   # (H-k+1, W-k+1, k, k)
    wb = np.lib.stride_tricks.sliding_window_view(b, (k, k))
    mu_a = np.einsum("yxuv,uv->yx", wa, w)
    mu_b = np.einsum("yxuv,uv->yx", wb, w)
    da = wa - mu_a[:, :, None, None]
    db = wb - mu_b[:, :, None, None]
    var_a = np.einsum("yxuv,uv->yx", da * da, w)
    var_b = np.einsum("yxuv,uv->yx", db * db, w)
    cov = np.einsum("yxuv,uv->yx", da * db, w)
    num = (2.0 * mu_a * mu_b + SSIM_C1) * (2.0 * cov + SSIM_C2)
    den = (mu_a * mu_a + mu_b * mu_b + SSIM_C1) * (var_a + var_b + SSIM_C2)
    return num / den


def ssim(a: np.ndarray, b: np.ndarray) -> float:
    """Mean SSIM over all window positions; NaN when the image is smaller than the window."""
    m = ssim_map(a, b)
    return float(m.mean()) if m.size else math.nan


def image_stats(a: np.ndarray, b: np.ndarray | None = None, with_ssim: bool = False) -> dict:
    """All statistics of one image (and of the pair, when b is given)."""
    a = np.asarray(a, dtype=np.uint8)
    out = {"hist": histogram(a), "entropy": entropy(a), "chi2": chi2(a)}
    if b is not None:
        b = np.asarray(b, dtype=np.uint8)
        d = np.abs(a.astype(np.int64) - b.astype(np.int64))
        out.update(n_diff=int(np.count_nonzero(d)), sum_abs=int(d.sum()), sum_sq=int((d * d).sum()),
                   npcr=npcr(a, b), uaci=uaci(a, b), psnr=psnr(a, b))
        if with_ssim:
            out["ssim"] = ssim(a, b)
    return out
