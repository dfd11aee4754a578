"""ctypes binding of the plain-C oracle (TEST INFRASTRUCTURE ONLY).

Each wrapper names the paper passage its C routine restates; see rdhei_oracle.c for
the literal steps.  No arithmetic of the method happens here: only array
allocation, packing of arguments and unpacking of results.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

EMR, LMR = 0, 1
# EMR / LMR with the MED predictor of the related work (Sec. II) instead of the glide
EMR_MED, LMR_MED = 2, 3
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rdhei_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc -O2 (no intrinsics, portable to x86 and Arm)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


_u8p = ctypes.POINTER(ctypes.c_uint8)
_u32p = ctypes.POINTER(ctypes.c_uint32)


def _declare(L):
    c = ctypes
    L.orc_keystream.argtypes = [_u8p, _u8p, c.c_uint64, _u8p]
    L.orc_chacha20_block.argtypes = [_u8p, c.c_uint32, _u8p, _u8p]
    L.orc_glide_labels.argtypes = [_u8p, c.c_int, c.c_int, c.c_int, _u8p]
    L.orc_label_hist.argtypes = [_u8p, c.c_int, c.c_int, _u32p]
    L.orc_med_labels.argtypes = [_u8p, c.c_int, c.c_int, c.c_int, c.c_int, _u8p]
    L.orc_med_hist.argtypes = [_u8p, c.c_int, c.c_int, c.c_int, _u32p]
    L.orc_choose_b.argtypes = [c.c_int, _u32p]
    L.orc_choose_b.restype = c.c_int
    L.orc_levels.argtypes = [c.c_int, c.c_int]
    L.orc_levels.restype = c.c_int
    L.orc_block_angle.argtypes = [_u8p, c.c_int, c.c_int, c.c_int, c.c_int, c.c_int]
    L.orc_block_angle.restype = c.c_int
    L.orc_rotate.argtypes = [c.POINTER(_u8p), c.c_int, c.c_int, c.c_int, _u8p, c.c_int, c.c_int]
    L.orc_effective_lmin.argtypes = [c.c_int, c.c_int, c.c_int, c.c_int]
    L.orc_effective_lmin.restype = c.c_int
    L.orc_label_encrypt.argtypes = [c.c_int, c.c_int, c.c_int, c.c_int, _u8p, _u8p, _u8p, c.c_int, c.c_int,
                                    _u8p, _u8p, _u8p, _u8p, c.c_uint64, _u32p, c.POINTER(c.c_int),
                                    c.POINTER(c.c_uint64)]
    L.orc_lmr_set_side.argtypes = [_u8p, c.c_uint64, _u8p, c.c_uint64]
    L.orc_embed.argtypes = [c.c_int, c.c_int, _u8p, _u8p, _u8p, c.c_int, c.c_int, _u8p, _u8p, c.c_uint64, _u8p]
    L.orc_embed.restype = c.c_uint64
    L.orc_extract.argtypes = [c.c_int, c.c_int, _u8p, _u8p, _u8p, c.c_int, c.c_int, _u8p, _u8p, c.c_uint64]
    L.orc_extract.restype = c.c_uint64
    L.orc_decrypt_recover.argtypes = [c.c_int, c.c_int, c.c_int, c.c_int, _u8p, _u8p, _u8p, c.c_int, c.c_int,
                                      _u8p, _u8p, _u8p]


def _p(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_u8p)


def _key(k, n):
    a = np.frombuffer(bytes(k), dtype=np.uint8).copy()
    assert a.size == n
    return a


def nbytes_for_bits(nbits: int) -> int:
    return (int(nbits) + 7) // 8


# ----------------------------------------------------------------------------------
# keystream (Sec. "Secret key generation"; ChaCha20 per RFC 8439)
# ----------------------------------------------------------------------------------
def keystream(key: bytes, nonce: bytes, nbytes: int) -> np.ndarray:
    out = np.zeros(max(int(nbytes), 1), np.uint8)
    k, n = _key(key, 32), _key(nonce, 12)
    lib().orc_keystream(_p(k), _p(n), int(nbytes), _p(out))
    return out[: int(nbytes)]


def chacha20_block(key: bytes, counter: int, nonce: bytes) -> np.ndarray:
    out = np.zeros(64, np.uint8)
    k, n = _key(key, 32), _key(nonce, 12)
    lib().orc_chacha20_block(_p(k), int(counter), _p(n), _p(out))
    return out


# ----------------------------------------------------------------------------------
# location maps, label histogram, b (Eqs. gliding1/2, optimal_b)
# ----------------------------------------------------------------------------------
def glide_labels(img: np.ndarray, b: int) -> np.ndarray:
    img = np.ascontiguousarray(img, np.uint8)
    H, W = img.shape
    out = np.zeros((H, W), np.uint8)
    lib().orc_glide_labels(_p(img), H, W, int(b), _p(out))
    return out


def label_hist(img: np.ndarray) -> np.ndarray:
    img = np.ascontiguousarray(img, np.uint8)
    H, W = img.shape
    h = np.zeros(9, np.uint32)
    lib().orc_label_hist(_p(img), H, W, h.ctypes.data_as(_u32p))
    return h


def med_labels(img: np.ndarray, b: int, seven: bool) -> np.ndarray:
    """b-MSB location map against the MED prediction (related work, Sec. II);
    seven: predict on the top seven bits (EMR layout)."""
    img = np.ascontiguousarray(img, np.uint8)
    H, W = img.shape
    out = np.zeros((H, W), np.uint8)
    lib().orc_med_labels(_p(img), H, W, int(bool(seven)), int(b), _p(out))
    return out


def med_hist(img: np.ndarray, seven: bool) -> np.ndarray:
    img = np.ascontiguousarray(img, np.uint8)
    H, W = img.shape
    h = np.zeros(9, np.uint32)
    lib().orc_med_hist(_p(img), H, W, int(bool(seven)), h.ctypes.data_as(_u32p))
    return h


def choose_b(variant: int, hist: np.ndarray) -> int:
    h = np.ascontiguousarray(hist, np.uint32)
    return int(lib().orc_choose_b(int(variant), h.ctypes.data_as(_u32p)))


# ----------------------------------------------------------------------------------
# rotation (Eqs. roration / roration2)
# ----------------------------------------------------------------------------------
def levels(H: int, W: int) -> int:
    return int(lib().orc_levels(H, W))


def effective_lmin(variant: int, lmin: int, H: int, W: int) -> int:
    return int(lib().orc_effective_lmin(variant, lmin, H, W))


def block_angle(s: np.ndarray, H: int, W: int, L: int, C1: int, C2: int) -> int:
    s = np.ascontiguousarray(s, np.uint8).reshape(-1)
    return int(lib().orc_block_angle(_p(s), H, W, L, C1, C2))


def rotate(planes, s: np.ndarray, lmin: int, direction: int):
    """Rotate copies of the given H x W uint8 planes; direction 0 encode, 1 decode."""
    planes = [np.ascontiguousarray(p, np.uint8).copy() for p in planes]
    H, W = planes[0].shape
    s = np.ascontiguousarray(s, np.uint8).reshape(-1)
    arr = (_u8p * len(planes))(*[_p(p) for p in planes])
    lib().orc_rotate(arr, len(planes), H, W, _p(s), int(lmin), int(direction))
    return planes


# ----------------------------------------------------------------------------------
# the four calls of the method
# ----------------------------------------------------------------------------------
@dataclass
class Params:
    variant: int = EMR
    b: int = 0               # 0 = Eq. optimal_b
    rot_lmin: int = 0        # 0 = variant default
    rot_enable: int = 1
    k1: bytes = bytes(32)
    nonce1: bytes = bytes(12)
    k2: bytes = bytes(32)
    nonce2: bytes = bytes(12)


@dataclass
class Encoded:
    enc: np.ndarray
    map_bits: np.ndarray
    eta_bits: np.ndarray
    hist: np.ndarray
    b: int
    capacity: int


def label_encrypt(p: Params, img: np.ndarray, side_bits: np.ndarray | None = None, side_nbits: int = 0) -> Encoded:
    img = np.ascontiguousarray(img, np.uint8)
    H, W = img.shape
    enc = np.zeros((H, W), np.uint8)
    nb = max(nbytes_for_bits(H * W), 1)
    mb, eb = np.zeros(nb, np.uint8), np.zeros(nb, np.uint8)
    hist = np.zeros(9, np.uint32)
    b_out, cap = ctypes.c_int(0), ctypes.c_uint64(0)
    side = None if side_bits is None else np.ascontiguousarray(side_bits, np.uint8)
    lib().orc_label_encrypt(p.variant, p.b, p.rot_lmin, p.rot_enable, _p(_key(p.k1, 32)), _p(_key(p.nonce1, 12)),
                            _p(img), H, W, _p(enc), _p(mb), _p(eb), _p(side), int(side_nbits),
                            hist.ctypes.data_as(_u32p), ctypes.byref(b_out), ctypes.byref(cap))
    return Encoded(enc, mb[: nbytes_for_bits(H * W)], eb[: nbytes_for_bits(H * W)], hist, b_out.value, cap.value)


def lmr_set_side(enc: np.ndarray, side_bits: np.ndarray, side_nbits: int) -> np.ndarray:
    out = np.ascontiguousarray(enc, np.uint8).copy()
    side = np.ascontiguousarray(side_bits, np.uint8)
    lib().orc_lmr_set_side(_p(out), out.size, _p(side), int(side_nbits))
    return out


def embed(p: Params, b: int, enc: np.ndarray, payload: np.ndarray, nbits: int, lmr_map: np.ndarray | None = None):
    enc = np.ascontiguousarray(enc, np.uint8)
    H, W = enc.shape
    marked = np.zeros_like(enc)
    pay = np.ascontiguousarray(payload, np.uint8)
    if pay.size == 0:
        pay = np.zeros(1, np.uint8)
    m = None if lmr_map is None else np.ascontiguousarray(lmr_map, np.uint8)
    k = lib().orc_embed(p.variant, int(b), _p(_key(p.k2, 32)), _p(_key(p.nonce2, 12)), _p(enc), H, W, _p(m),
                        _p(pay), int(nbits), _p(marked))
    return marked, int(k)


def extract(p: Params, b: int, marked: np.ndarray, max_bits: int, lmr_map: np.ndarray | None = None):
    marked = np.ascontiguousarray(marked, np.uint8)
    H, W = marked.shape
    out = np.zeros(max(nbytes_for_bits(max_bits), 1), np.uint8)
    m = None if lmr_map is None else np.ascontiguousarray(lmr_map, np.uint8)
    k = lib().orc_extract(p.variant, int(b), _p(_key(p.k2, 32)), _p(_key(p.nonce2, 12)), _p(marked), H, W, _p(m),
                          _p(out), int(max_bits))
    return out[: nbytes_for_bits(k)], int(k)


def decrypt_recover(p: Params, b: int, marked: np.ndarray, lmr_map: np.ndarray | None = None,
                    lmr_eta: np.ndarray | None = None) -> np.ndarray:
    marked = np.ascontiguousarray(marked, np.uint8)
    H, W = marked.shape
    out = np.zeros_like(marked)
    m = None if lmr_map is None else np.ascontiguousarray(lmr_map, np.uint8)
    e = None if lmr_eta is None else np.ascontiguousarray(lmr_eta, np.uint8)
    lib().orc_decrypt_recover(p.variant, int(b), p.rot_lmin, p.rot_enable, _p(_key(p.k1, 32)),
                              _p(_key(p.nonce1, 12)), _p(marked), H, W, _p(m), _p(e), _p(out))
    return out
