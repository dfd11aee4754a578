"""Seeded synthetic inputs: 8-bit grayscale images, payload bits, keys.

This module holds none of the method's arithmetic; it only draws inputs.  The paper
measures on the BOWS-2 set and standard 512 x 512 test images (Sec. IV), which are not
available here; these images stand in for them with the same size and bit depth and
natural-image-like local smoothness:

  base 128
  + 8 plane sinusoids  A sin(2 pi (fx x / W + fy y / H) + phi),  A ~ U[8, 32],
                       fx, fy ~ U[-4, 4] cycles per image, phi ~ U[0, 2 pi)
  + n_blobs isotropic Gaussian blobs, amplitude ~ U[-64, 64],
                       sigma ~ U[0.02, 0.15] * min(H, W), centres uniform
  + Gaussian texture noise N(0, sigma_n)
  then round half to even and clip to 0..255.

Sinusoids and blobs are separable (angle-addition / product of 1-D Gaussians), so
they are evaluated as outer products and even 8192 x 8192 images are cheap.
Image k of a set with base seed S uses ``seed = S * 1_000_003 + k``; its payload bits
come from ``default_rng(seed ^ 0x9E3779B9)``; its keys are SHA-256 digests of
("k1" | "k2") + seed, and its nonces encode the image index.
"""
from __future__ import annotations

import hashlib

import numpy as np

SEED_STRIDE = 1_000_003
PAYLOAD_SALT = 0x9E3779B9


def image_seed(base_seed: int, k: int) -> int:
    return int(base_seed) * SEED_STRIDE + int(k)


def synth_image(H: int, W: int, seed: int, n_blobs: int = 16, noise_sigma: float = 4.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    x = np.arange(W, dtype=np.float64)
    y = np.arange(H, dtype=np.float64)
    img = np.full((H, W), 128.0)
    for _ in range(8):
        A = rng.uniform(8, 32)
        fx, fy = rng.uniform(-4, 4), rng.uniform(-4, 4)
        phi = rng.uniform(0, 2 * np.pi)
        ax = 2 * np.pi * fx * x / W + phi
        ay = 2 * np.pi * fy * y / H
        # sin(ay + ax) = sin(ay) cos(ax) + cos(ay) sin(ax)
        img += A * (np.outer(np.sin(ay), np.cos(ax)) + np.outer(np.cos(ay), np.sin(ax)))
    m = min(H, W)
    for _ in range(int(n_blobs)):
        amp = rng.uniform(-64, 64)
        sig = rng.uniform(0.02, 0.15) * m
        cx, cy = rng.uniform(0, W), rng.uniform(0, H)
        gx = np.exp(-((x - cx) ** 2) / (2 * sig * sig))
        gy = np.exp(-((y - cy) ** 2) / (2 * sig * sig))
        img += amp * np.outer(gy, gx)
    img += rng.normal(0.0, noise_sigma, size=(H, W))
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def batch_image(base_seed: int, k: int, H: int = 512, W: int = 512, vary: bool = True) -> np.ndarray:
    """Image k of a batch; with ``vary`` the smoothness is drawn per image
    (noise sigma ~ U[1, 16], blob count ~ U{4..64})."""
    seed = image_seed(base_seed, k)
    if vary:
        r = np.random.default_rng(seed ^ 0x5DEECE66D)
        sigma = r.uniform(1, 16)
        blobs = int(r.integers(4, 65))
    else:
        sigma, blobs = 4.0, 16
    return synth_image(H, W, seed, n_blobs=blobs, noise_sigma=sigma)


def payload_bits(seed: int, nbits: int) -> np.ndarray:
    """nbits random payload bits packed MSB-first into ceil(nbits/8) bytes."""
    rng = np.random.default_rng(int(seed) ^ PAYLOAD_SALT)
    nbytes = (int(nbits) + 7) // 8
    out = rng.integers(0, 256, size=nbytes, dtype=np.uint8)
    if nbits % 8:
        out[-1] &= np.uint8((0xFF << (8 - nbits % 8)) & 0xFF)
    return out


def keys(seed: int) -> dict:
    s = str(int(seed)).encode()
    return {
        "k1": hashlib.sha256(b"k1" + s).digest(),
        "k2": hashlib.sha256(b"k2" + s).digest(),
        "nonce1": int(seed % (1 << 64)).to_bytes(8, "little") + b"\x01\x00\x00\x00",
        "nonce2": int(seed % (1 << 64)).to_bytes(8, "little") + b"\x02\x00\x00\x00",
    }


def random_bits(seed: int, nbits: int) -> np.ndarray:
    """Stand-in bit stream (e.g. the LMR side information when no compressor runs)."""
    return payload_bits(seed ^ 0x51DE, nbits)
