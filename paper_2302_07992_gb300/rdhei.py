"""Thin ctypes binding of ``librdhei.so`` (C ABI in ``include/rdhei.h``).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.  Importing this module loads
the library and fails loudly if it has not been built (``python -m
paper_2302_07992_gb300.build``) -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import torch

from . import build as _build

EMR, LMR = 0, 1
# the related-work variants: MED (LOCO-I) prediction instead of the paper's glide
EMR_MED, LMR_MED = 2, 3
OP_LABEL_ENCRYPT, OP_EMBED, OP_EXTRACT, OP_DECRYPT_RECOVER, OP_LMR_SET_SIDE = 0, 1, 2, 3, 4
# fused calls: owner + hider, and the receiver with both keys
OP_ENCODE, OP_DECODE = 5, 6
STATUS = {0: "OK", 1: "EINVAL", 2: "ECAPACITY", 3: "ECUDA", 4: "ETIMEOUT", 5: "ESPACE", 6: "EBOUNDS"}
RDHEI_OK, RDHEI_EINVAL, RDHEI_ECAPACITY, RDHEI_ECUDA, RDHEI_ETIMEOUT, RDHEI_ESPACE, RDHEI_EBOUNDS = range(7)
RDHEI_BUILD_CHECKED = 1

# RDHEI_CHECKED=1 selects the checked build (device index checks, RDHEI_EBOUNDS)
LIBRARY = _build.LIB_CHECKED if os.environ.get("RDHEI_CHECKED", "0") == "1" else _build.LIB
if not os.path.exists(LIBRARY):
    raise ImportError(f"{LIBRARY} is missing: build it with `python -m paper_2302_07992_gb300.build` "
                      "(add --checked for the checked build, or __graft_entry__.build()); "
                      "there is no CPU fallback")
_lib = ctypes.CDLL(LIBRARY)


class Job(ctypes.Structure):
    _fields_ = [
        ("H", ctypes.c_int32), ("W", ctypes.c_int32), ("variant", ctypes.c_int32), ("b", ctypes.c_int32),
        ("rot_lmin", ctypes.c_int32), ("rot_enable", ctypes.c_int32),
        ("k1", ctypes.c_uint8 * 32), ("nonce1", ctypes.c_uint8 * 12),
        ("k2", ctypes.c_uint8 * 32), ("nonce2", ctypes.c_uint8 * 12),
        ("src", ctypes.c_void_p), ("dst", ctypes.c_void_p), ("map_bits", ctypes.c_void_p),
        ("eta_bits", ctypes.c_void_p), ("side_bits", ctypes.c_void_p), ("side_nbits", ctypes.c_uint64),
        ("payload", ctypes.c_void_p), ("nbits", ctypes.c_uint64),
        ("bits_out", ctypes.c_void_p), ("max_bits", ctypes.c_uint64),
        ("info", ctypes.c_void_p),
    ]


class Info(ctypes.Structure):
    _fields_ = [("hist", ctypes.c_uint32 * 9), ("b", ctypes.c_int32), ("capacity", ctypes.c_uint64),
                ("embedded", ctypes.c_uint64), ("extracted", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


INFO_BYTES = ctypes.sizeof(Info)

_JobP = ctypes.POINTER(Job)
_lib.rdhei_workspace_size.argtypes = [_JobP, ctypes.c_int]
_lib.rdhei_workspace_size.restype = ctypes.c_size_t
for _n in ("rdhei_label_encrypt", "rdhei_embed", "rdhei_extract", "rdhei_decrypt_recover", "rdhei_lmr_set_side",
           "rdhei_encode", "rdhei_decode"):
    getattr(_lib, _n).argtypes = [_JobP, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    getattr(_lib, _n).restype = ctypes.c_int
_lib.rdhei_plan_create.argtypes = [_JobP, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
_lib.rdhei_plan_create.restype = ctypes.c_int
_lib.rdhei_plan_workspace_size.argtypes = [ctypes.c_void_p]
_lib.rdhei_plan_workspace_size.restype = ctypes.c_size_t
_lib.rdhei_plan_upload.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
_lib.rdhei_plan_upload.restype = ctypes.c_int
_lib.rdhei_plan_staging_size.argtypes = [ctypes.c_void_p]
_lib.rdhei_plan_staging_size.restype = ctypes.c_size_t
_lib.rdhei_plan_upload_async.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                         ctypes.c_size_t, ctypes.c_void_p]
_lib.rdhei_plan_upload_async.restype = ctypes.c_int
_lib.rdhei_plan_run.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
_lib.rdhei_plan_run.restype = ctypes.c_int
_lib.rdhei_plan_run_stage.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
_lib.rdhei_plan_run_stage.restype = ctypes.c_int
_lib.rdhei_plan_stage_count.argtypes = [ctypes.c_int]
_lib.rdhei_plan_stage_count.restype = ctypes.c_int
_lib.rdhei_stage_name.argtypes = [ctypes.c_int, ctypes.c_int]
_lib.rdhei_stage_name.restype = ctypes.c_char_p
_lib.rdhei_plan_stage_active.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
_lib.rdhei_plan_stage_active.restype = ctypes.c_int
_lib.rdhei_plan_set_wave_cols.argtypes = [ctypes.c_void_p, ctypes.c_int]
_lib.rdhei_plan_set_wave_cols.restype = ctypes.c_int
_lib.rdhei_plan_set_param.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
_lib.rdhei_plan_set_param.restype = ctypes.c_int
_lib.rdhei_plan_get_param.argtypes = [ctypes.c_void_p, ctypes.c_int]
_lib.rdhei_plan_get_param.restype = ctypes.c_int
PARAM_WAVE_COLS, PARAM_EXTRACT_ROWS, PARAM_ENC_SPLIT = 1, 2, 3
_lib.rdhei_plan_destroy.argtypes = [ctypes.c_void_p]
_lib.rdhei_plan_destroy.restype = None
_lib.rdhei_workspace_status.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]
_lib.rdhei_workspace_status.restype = ctypes.c_int
_lib.rdhei_job_size.restype = ctypes.c_size_t
_lib.rdhei_info_size.restype = ctypes.c_size_t
_lib.rdhei_version.restype = ctypes.c_char_p
_lib.rdhei_build_flags.argtypes = []
_lib.rdhei_build_flags.restype = ctypes.c_int
_lib.rdhei_plan_copy_status.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
_lib.rdhei_plan_copy_status.restype = ctypes.c_int
_lib.rdhei_wait_selftest.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
_lib.rdhei_wait_selftest.restype = ctypes.c_int

assert _lib.rdhei_job_size() == ctypes.sizeof(Job), "rdhei_job layout mismatch"
assert _lib.rdhei_info_size() == ctypes.sizeof(Info), "rdhei_info layout mismatch"


class RdheiError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != 0:
        raise RdheiError(f"{what} failed: {STATUS.get(rc, rc)}")


def version() -> str:
    return _lib.rdhei_version().decode()


def wait_selftest(flag: torch.Tensor, limit_ns: int, stream=None) -> int:
    """Bounded-wait self-test: waits on the device word flag[0] for at most limit_ns
    and returns the status the kernel wrote (RDHEI_OK or RDHEI_ETIMEOUT)."""
    assert flag.is_cuda and flag.dtype in (torch.int32, torch.uint32) and flag.numel() >= 1
    status = torch.full((1,), -1, dtype=torch.int32, device=flag.device)
    _check(_lib.rdhei_wait_selftest(ctypes.c_void_p(flag.data_ptr()), int(limit_ns),
                                    ctypes.c_void_p(status.data_ptr()), _stream(stream)), "rdhei_wait_selftest")
    return int(status.item())


def checked() -> bool:
    """True when the loaded library is the checked build (device index checks)."""
    return bool(_lib.rdhei_build_flags() & RDHEI_BUILD_CHECKED)


def stages(op: int) -> list[str]:
    """Names of the kernels one operation launches, in launch order."""
    return [_lib.rdhei_stage_name(op, s).decode() for s in range(_lib.rdhei_plan_stage_count(op))]


def library_path() -> str:
    return _build.LIB


# ----------------------------------------------------------------------------------
@dataclass
class Params:
    """Per-image method parameters (mirrors the job fields of include/rdhei.h)."""
    variant: int = EMR
    b: int = 0
    rot_lmin: int = 0
    rot_enable: int = 1
    k1: bytes = bytes(32)
    nonce1: bytes = bytes(12)
    k2: bytes = bytes(32)
    nonce2: bytes = bytes(12)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def bitbuf(nbits: int, device="cuda") -> torch.Tensor:
    """Zeroed device buffer for an nbits stream, padded to whole 32-bit words."""
    return torch.zeros(max(4, ((int(nbits) + 31) // 32) * 4), dtype=torch.uint8, device=device)


def as_bitbuf(packed: torch.Tensor, nbits: int) -> torch.Tensor:
    """Copy an MSB-first packed stream into a word-padded device buffer."""
    out = bitbuf(nbits, packed.device if packed.is_cuda else "cuda")
    n = min(packed.numel(), out.numel())
    out[:n].copy_(packed.reshape(-1)[:n])
    return out


def make_job(p: Params, H: int, W: int, *, src=None, dst=None, map_bits=None, eta_bits=None, side_bits=None,
             side_nbits=0, payload=None, nbits=0, bits_out=None, max_bits=0, info=None, b=None) -> Job:
    j = Job()
    j.H, j.W, j.variant = int(H), int(W), int(p.variant)
    j.b = int(p.b if b is None else b)
    j.rot_lmin, j.rot_enable = int(p.rot_lmin), int(p.rot_enable)
    for name, n in (("k1", 32), ("nonce1", 12), ("k2", 32), ("nonce2", 12)):
        v = bytes(getattr(p, name))
        assert len(v) == n, name
        ctypes.memmove(ctypes.addressof(getattr(j, name)), v, n)
    j.src, j.dst = _ptr(src), _ptr(dst)
    j.map_bits, j.eta_bits, j.side_bits = _ptr(map_bits), _ptr(eta_bits), _ptr(side_bits)
    j.side_nbits = int(side_nbits)
    j.payload, j.nbits = _ptr(payload), int(nbits)
    j.bits_out, j.max_bits = _ptr(bits_out), int(max_bits)
    j.info = _ptr(info)
    return j


def new_info(n: int = 1, device="cuda") -> torch.Tensor:
    return torch.zeros((n, INFO_BYTES), dtype=torch.uint8, device=device)


def read_info(info: torch.Tensor) -> list[dict]:
    host = info.detach().to("cpu").contiguous()
    out = []
    for i in range(host.shape[0]):
        raw = bytes(host[i].numpy().tobytes())
        s = Info.from_buffer_copy(raw)
        out.append({"hist": list(s.hist), "b": s.b, "capacity": s.capacity, "embedded": s.embedded,
                    "extracted": s.extracted, "status": s.status})
    return out


class Plan:
    """A validated, uploaded batch: ``run(op)`` launches kernels only (capturable)."""

    def __init__(self, jobs: list[Job], stream=None, workspace: torch.Tensor | None = None,
                 wave_cols: int | None = None, params: dict | None = None, staging=None):
        """staging: a callable nbytes -> page-locked uint8 host tensor; when given, the
        descriptors go up asynchronously from it (rdhei_plan_upload_async) and the
        caller keeps self.staging alive until the stream has passed the upload."""
        self._jobs = (Job * len(jobs))(*jobs)
        h = ctypes.c_void_p()
        _check(_lib.rdhei_plan_create(self._jobs, len(jobs), ctypes.byref(h)), "rdhei_plan_create")
        self._h = h
        if wave_cols is not None:
            _check(_lib.rdhei_plan_set_wave_cols(h, int(wave_cols)), "rdhei_plan_set_wave_cols")
        for k, v in (params or {}).items():
            self.set_param(k, v)
        self.wave_cols = wave_cols
        need = _lib.rdhei_plan_workspace_size(h)
        if workspace is None or workspace.numel() < need:
            workspace = torch.empty(max(int(need), 256) + 256, dtype=torch.uint8, device="cuda")
        self.ws = workspace
        off = (-self.ws.data_ptr()) % 256
        self._ws_ptr = self.ws.data_ptr() + off
        self._ws_bytes = self.ws.numel() - off
        self.staging = None
        if staging is None:
            _check(_lib.rdhei_plan_upload(h, ctypes.c_void_p(self._ws_ptr), self._ws_bytes, _stream(stream)),
                   "rdhei_plan_upload")
        else:
            nb = int(_lib.rdhei_plan_staging_size(h))
            self.staging = staging(max(nb, 16))
            _check(_lib.rdhei_plan_upload_async(h, ctypes.c_void_p(self._ws_ptr), self._ws_bytes,
                                                ctypes.c_void_p(self.staging.data_ptr()), self.staging.numel(),
                                                _stream(stream)), "rdhei_plan_upload_async")

    def run(self, op: int, stream=None):
        _check(_lib.rdhei_plan_run(self._h, int(op), _stream(stream)), f"rdhei_plan_run({op})")

    def run_stage(self, op: int, stage: int, stream=None):
        _check(_lib.rdhei_plan_run_stage(self._h, int(op), int(stage), _stream(stream)),
               f"rdhei_plan_run_stage({op}, {stage})")

    def set_param(self, param: int, value: int):
        """A free launch parameter (PARAM_*); results do not depend on it."""
        _check(_lib.rdhei_plan_set_param(self._h, int(param), int(value)), f"rdhei_plan_set_param({param})")

    def get_param(self, param: int) -> int:
        return int(_lib.rdhei_plan_get_param(self._h, int(param)))

    def active_stages(self, op: int) -> list[int]:
        """Stages of op that launch work for this plan's jobs."""
        return [s for s in range(len(stages(op))) if _lib.rdhei_plan_stage_active(self._h, int(op), s)]

    def copy_status(self, dst: torch.Tensor, stream=None):
        """Queue a copy of the workspace error word into dst (an int32 element of
        pinned host or device memory) behind this plan's work on `stream`; status()
        reads it synchronously instead."""
        assert dst.dtype == torch.int32 and dst.numel() >= 1 and (dst.is_cuda or dst.is_pinned())
        _check(_lib.rdhei_plan_copy_status(self._h, ctypes.c_void_p(dst.data_ptr()), _stream(stream)),
               "rdhei_plan_copy_status")

    def status(self, stream=None) -> int:
        code = ctypes.c_int32(0)
        _check(_lib.rdhei_workspace_status(ctypes.c_void_p(self._ws_ptr), _stream(stream), ctypes.byref(code)),
               "rdhei_workspace_status")
        return int(code.value)

    def close(self):
        if getattr(self, "_h", None):
            _lib.rdhei_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_jobs(op: int, jobs: list[Job], stream=None, check: bool = True) -> int:
    """One call of the C ABI's named entry point for ``op`` on a batch of jobs."""
    arr = (Job * len(jobs))(*jobs)
    need = _lib.rdhei_workspace_size(arr, len(jobs))
    if need == 0:
        raise RdheiError("rdhei_workspace_size rejected the jobs")
    ws = torch.empty(int(need) + 256, dtype=torch.uint8, device="cuda")
    off = (-ws.data_ptr()) % 256
    fn = {OP_LABEL_ENCRYPT: _lib.rdhei_label_encrypt, OP_EMBED: _lib.rdhei_embed, OP_EXTRACT: _lib.rdhei_extract,
          OP_DECRYPT_RECOVER: _lib.rdhei_decrypt_recover, OP_LMR_SET_SIDE: _lib.rdhei_lmr_set_side,
          OP_ENCODE: _lib.rdhei_encode, OP_DECODE: _lib.rdhei_decode}[op]
    st = _stream(stream)
    _check(fn(arr, len(jobs), ctypes.c_void_p(ws.data_ptr() + off), ws.numel() - off, st), f"op {op}")
    code = ctypes.c_int32(0)
    _check(_lib.rdhei_workspace_status(ctypes.c_void_p(ws.data_ptr() + off), st, ctypes.byref(code)),
           "rdhei_workspace_status")
    if check and code.value not in (0, 2):
        raise RdheiError(f"device reported {STATUS.get(code.value, code.value)}")
    return int(code.value)


# ---------------------------------------------------------------- one image --
def label_encrypt(img: torch.Tensor, p: Params, side_bits: torch.Tensor | None = None, side_nbits: int = 0,
                  want_maps: bool = True, info: torch.Tensor | None = None, stream=None) -> dict:
    H, W = img.shape
    img = img.contiguous()
    enc = torch.empty_like(img)
    info = new_info(1) if info is None else info
    mb = bitbuf(H * W) if want_maps else None
    eb = bitbuf(H * W) if (want_maps and (p.variant & 1) == LMR) else None
    sb = None if side_bits is None else as_bitbuf(side_bits, side_nbits)
    j = make_job(p, H, W, src=img, dst=enc, map_bits=mb, eta_bits=eb, side_bits=sb, side_nbits=side_nbits,
                 info=info)
    run_jobs(OP_LABEL_ENCRYPT, [j], stream)
    return {"enc": enc, "map_bits": mb, "eta_bits": eb, "info": info, **read_info(info)[0]}


def embed(enc: torch.Tensor, p: Params, b: int, payload: torch.Tensor, nbits: int,
          lmr_map: torch.Tensor | None = None, info: torch.Tensor | None = None, stream=None) -> dict:
    H, W = enc.shape
    out = torch.empty_like(enc)
    info = new_info(1) if info is None else info
    pay = as_bitbuf(payload, nbits)
    j = make_job(p, H, W, src=enc.contiguous(), dst=out, map_bits=lmr_map, payload=pay, nbits=nbits, info=info, b=b)
    code = run_jobs(OP_EMBED, [j], stream)
    return {"marked": out, "status": code, **read_info(info)[0]}


def extract(marked: torch.Tensor, p: Params, b: int, max_bits: int, lmr_map: torch.Tensor | None = None,
            info: torch.Tensor | None = None, stream=None) -> dict:
    H, W = marked.shape
    info = new_info(1) if info is None else info
    out = bitbuf(max_bits)
    j = make_job(p, H, W, src=marked.contiguous(), map_bits=lmr_map, bits_out=out, max_bits=max_bits, info=info,
                 b=b)
    run_jobs(OP_EXTRACT, [j], stream)
    r = read_info(info)[0]
    return {"bits": out, **r}


def decrypt_recover(marked: torch.Tensor, p: Params, b: int, lmr_map: torch.Tensor | None = None,
                    lmr_eta: torch.Tensor | None = None, info: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    H, W = marked.shape
    info = new_info(1) if info is None else info
    out = torch.empty_like(marked)
    j = make_job(p, H, W, src=marked.contiguous(), dst=out, map_bits=lmr_map, eta_bits=lmr_eta, info=info, b=b)
    run_jobs(OP_DECRYPT_RECOVER, [j], stream)
    return out


def encode(img: torch.Tensor, p: Params, payload: torch.Tensor, nbits: int, side_bits: torch.Tensor | None = None,
           side_nbits: int = 0, info: torch.Tensor | None = None, stream=None) -> dict:
    """rdhei_encode: the owner's label_encrypt and the hider's embed in one call."""
    H, W = img.shape
    out = torch.empty_like(img)
    info = new_info(1) if info is None else info
    lmr = (p.variant & 1) == LMR
    mb = bitbuf(H * W)
    eb = bitbuf(H * W) if lmr else None
    sb = None if side_bits is None else as_bitbuf(side_bits, side_nbits)
    pay = as_bitbuf(payload, nbits)
    j = make_job(p, H, W, src=img.contiguous(), dst=out, map_bits=mb, eta_bits=eb, side_bits=sb,
                 side_nbits=side_nbits, payload=pay, nbits=nbits, info=info)
    code = run_jobs(OP_ENCODE, [j], stream)
    return {"marked": out, "map_bits": mb, "eta_bits": eb, "status": code, "info": info, **read_info(info)[0]}


def decode(marked: torch.Tensor, p: Params, b: int, max_bits: int, lmr_map: torch.Tensor | None = None,
           lmr_eta: torch.Tensor | None = None, info: torch.Tensor | None = None, stream=None) -> dict:
    """rdhei_decode: the receiver with both keys (extract and decrypt_recover in one call)."""
    H, W = marked.shape
    info = new_info(1) if info is None else info
    out = torch.empty_like(marked)
    bits = bitbuf(max_bits)
    j = make_job(p, H, W, src=marked.contiguous(), dst=out, map_bits=lmr_map, eta_bits=lmr_eta, bits_out=bits,
                 max_bits=max_bits, info=info, b=b)
    run_jobs(OP_DECODE, [j], stream)
    return {"bits": bits, "recovered": out, **read_info(info)[0]}


def lmr_set_side(enc: torch.Tensor, p: Params, side_bits: torch.Tensor, side_nbits: int, stream=None) -> torch.Tensor:
    H, W = enc.shape
    out = enc.clone()
    info = new_info(1)
    j = make_job(p, H, W, dst=out, side_bits=as_bitbuf(side_bits, side_nbits), side_nbits=side_nbits, info=info)
    run_jobs(OP_LMR_SET_SIDE, [j], stream)
    return out


# ------------------------------------------------------- allocation-free extract --
_lib.rdhei_extract_noalloc.argtypes = [_JobP, ctypes.c_void_p]
_lib.rdhei_extract_noalloc.restype = ctypes.c_int
NOALLOC_MAX_PIXELS = 1 << 24


def extract_noalloc_job(job: Job, stream=None) -> int:
    """rdhei_extract_noalloc on one prepared job; returns the C status code.  For
    callers that cannot allocate device memory: the library uses a static device
    array instead of a workspace (one image, at most NOALLOC_MAX_PIXELS pixels)."""
    return int(_lib.rdhei_extract_noalloc(ctypes.byref(job), _stream(stream)))


# ------------------------------------------------------------- measurement probes --
_lib.rdhei_probe_alu.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
_lib.rdhei_probe_alu.restype = ctypes.c_int
_lib.rdhei_probe_keystream.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _JobP, ctypes.c_void_p,
                                       ctypes.c_void_p]
_lib.rdhei_probe_keystream.restype = ctypes.c_int
_lib.rdhei_probe_workspace_size.restype = ctypes.c_size_t
PROBE_THREADS, PROBE_ALU_OPS_PER_ITER = 256, 16


def probe_alu(out: torch.Tensor, blocks: int, iters: int, stream=None):
    """Launch the integer/logic-pipe probe: blocks * 256 threads * iters * 16 ALU ops."""
    assert out.is_cuda and out.numel() * out.element_size() >= 4 * blocks * PROBE_THREADS
    _check(_lib.rdhei_probe_alu(ctypes.c_void_p(out.data_ptr()), int(blocks), int(iters), _stream(stream)),
           "rdhei_probe_alu")


class KeystreamProbe:
    """The ChaCha20 keystream probe: blocks * 256 threads * per_thread blocks of 64 bytes."""

    def __init__(self, p: Params, device="cuda"):
        self.job = make_job(p, 1, 1)
        self.ws = torch.empty(int(_lib.rdhei_probe_workspace_size()) + 64, dtype=torch.uint8, device=device)
        self.ws_ptr = self.ws.data_ptr() + ((-self.ws.data_ptr()) % 16)

    def launch(self, out: torch.Tensor, blocks: int, per_thread: int, stream=None):
        assert out.is_cuda and out.numel() * out.element_size() >= 4 * blocks * PROBE_THREADS
        _check(_lib.rdhei_probe_keystream(ctypes.c_void_p(out.data_ptr()), int(blocks), int(per_thread),
                                          ctypes.byref(self.job), ctypes.c_void_p(self.ws_ptr), _stream(stream)),
               "rdhei_probe_keystream")


# ------------------------------------------------------ security statistics --
STATS_SSIM = 1


class StatsJob(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("W", ctypes.c_int32), ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("a", ctypes.c_void_p), ("b", ctypes.c_void_p), ("out", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("hist", ctypes.c_uint32 * 256), ("n_diff", ctypes.c_uint64), ("sum_abs", ctypes.c_uint64),
                ("sum_sq", ctypes.c_uint64), ("entropy", ctypes.c_double), ("chi2", ctypes.c_double),
                ("npcr", ctypes.c_double), ("uaci", ctypes.c_double), ("psnr", ctypes.c_double),
                ("ssim", ctypes.c_double)]


STATS_BYTES = ctypes.sizeof(Stats)
_StatsJobP = ctypes.POINTER(StatsJob)
_lib.rdhei_stats_workspace_size.argtypes = [_StatsJobP, ctypes.c_int]
_lib.rdhei_stats_workspace_size.restype = ctypes.c_size_t
_lib.rdhei_image_stats.argtypes = [_StatsJobP, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
_lib.rdhei_image_stats.restype = ctypes.c_int
_lib.rdhei_stats_size.restype = ctypes.c_size_t
_lib.rdhei_stats_job_size.restype = ctypes.c_size_t
assert _lib.rdhei_stats_size() == STATS_BYTES, "rdhei_stats layout mismatch"
assert _lib.rdhei_stats_job_size() == ctypes.sizeof(StatsJob), "rdhei_stats_job layout mismatch"


def stats_job(a: torch.Tensor, b: torch.Tensor | None, out: torch.Tensor, ssim: bool = False) -> StatsJob:
    """Job for one image (and its comparison image b); ``out`` is STATS_BYTES of device memory."""
    H, W = a.shape
    if b is not None:
        assert tuple(b.shape) == (H, W)
    j = StatsJob()
    j.H, j.W, j.flags = int(H), int(W), STATS_SSIM if ssim else 0
    j.a, j.b, j.out = _ptr(a), _ptr(b), _ptr(out)
    return j


def new_stats(n: int = 1, device="cuda") -> torch.Tensor:
    return torch.zeros((n, STATS_BYTES), dtype=torch.uint8, device=device)


def read_stats(out: torch.Tensor) -> list[dict]:
    host = out.detach().to("cpu").contiguous()
    res = []
    for i in range(host.shape[0]):
        s = Stats.from_buffer_copy(bytes(host[i].numpy().tobytes()))
        res.append({"hist": list(s.hist), "n_diff": s.n_diff, "sum_abs": s.sum_abs, "sum_sq": s.sum_sq,
                    "entropy": s.entropy, "chi2": s.chi2, "npcr": s.npcr, "uaci": s.uaci, "psnr": s.psnr,
                    "ssim": s.ssim})
    return res


_lib.rdhei_stats_plan_create.argtypes = [_StatsJobP, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_void_p)]
_lib.rdhei_stats_plan_create.restype = ctypes.c_int
_lib.rdhei_stats_plan_run.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
_lib.rdhei_stats_plan_run.restype = ctypes.c_int
_lib.rdhei_stats_plan_run_stage.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
_lib.rdhei_stats_plan_run_stage.restype = ctypes.c_int
_lib.rdhei_stats_plan_destroy.argtypes = [ctypes.c_void_p]
_lib.rdhei_stats_plan_destroy.restype = None
STATS_STAGES = ("stats_hist_pairs", "stats_ssim")


class StatsCall:
    """A stats plan: jobs validated and uploaded once (host-synchronous); ``run``
    launches the memset and kernels only, so it can be timed per stage or captured."""

    def __init__(self, jobs: list[StatsJob], stream=None):
        self._jobs = (StatsJob * len(jobs))(*jobs)
        self.n = len(jobs)
        need = _lib.rdhei_stats_workspace_size(self._jobs, self.n)
        if self.n and need == 0:
            raise RdheiError("rdhei_stats_workspace_size rejected the jobs")
        self._ws = torch.empty(int(need) + 256, dtype=torch.uint8, device="cuda")
        off = (-self._ws.data_ptr()) % 256
        h = ctypes.c_void_p()
        _check(_lib.rdhei_stats_plan_create(self._jobs, self.n, ctypes.c_void_p(self._ws.data_ptr() + off),
                                            self._ws.numel() - off, _stream(stream), ctypes.byref(h)),
               "rdhei_stats_plan_create")
        self._h = h

    def run(self, stream=None):
        _check(_lib.rdhei_stats_plan_run(self._h, _stream(stream)), "rdhei_stats_plan_run")

    def run_stage(self, stage: int, stream=None):
        _check(_lib.rdhei_stats_plan_run_stage(self._h, int(stage), _stream(stream)), "rdhei_stats_plan_run_stage")

    def close(self):
        if getattr(self, "_h", None):
            _lib.rdhei_stats_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def image_stats_once(jobs: list[StatsJob], stream=None):
    """rdhei_image_stats: validate, upload and launch in one call (workspace freed after)."""
    arr = (StatsJob * len(jobs))(*jobs)
    need = _lib.rdhei_stats_workspace_size(arr, len(jobs))
    if jobs and need == 0:
        raise RdheiError("rdhei_stats_workspace_size rejected the jobs")
    ws = torch.empty(int(need) + 256, dtype=torch.uint8, device="cuda")
    off = (-ws.data_ptr()) % 256
    _check(_lib.rdhei_image_stats(arr, len(jobs), ctypes.c_void_p(ws.data_ptr() + off), ws.numel() - off,
                                  _stream(stream)), "rdhei_image_stats")


def image_stats(pairs, ssim: bool = False, stream=None) -> list[dict]:
    """Statistics of each (a, b) pair of device uint8 images (b may be None), in one call."""
    out = new_stats(len(pairs))
    call = StatsCall([stats_job(a, b, out[i], ssim) for i, (a, b) in enumerate(pairs)])
    call.run(stream)
    return read_stats(out)


# ------------------------------------------------- LMR side information (host) --
class SidePackJob(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("W", ctypes.c_int32), ("b", ctypes.c_int32), ("status", ctypes.c_int32),
                ("eta_bits", ctypes.c_void_p), ("map_bits", ctypes.c_void_p), ("side", ctypes.c_void_p),
                ("side_nbits", ctypes.c_uint64)]


class SideUnpackJob(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("W", ctypes.c_int32), ("b", ctypes.c_int32), ("status", ctypes.c_int32),
                ("plane", ctypes.c_void_p), ("eta_bits", ctypes.c_void_p), ("map_bits", ctypes.c_void_p)]


_lib.rdhei_bilevel_encode.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                      ctypes.POINTER(ctypes.c_size_t)]
_lib.rdhei_bilevel_encode.restype = ctypes.c_int
_lib.rdhei_bilevel_decode.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
_lib.rdhei_bilevel_decode.restype = ctypes.c_int
_lib.rdhei_lmr_side_pack.argtypes = [ctypes.POINTER(SidePackJob), ctypes.c_int, ctypes.c_int]
_lib.rdhei_lmr_side_pack.restype = ctypes.c_int
_lib.rdhei_lmr_side_unpack.argtypes = [ctypes.POINTER(SideUnpackJob), ctypes.c_int, ctypes.c_int]
_lib.rdhei_lmr_side_unpack.restype = ctypes.c_int
_lib.rdhei_msb_plane.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
_lib.rdhei_msb_plane.restype = ctypes.c_int
_lib.rdhei_side_pack_job_size.restype = ctypes.c_size_t
_lib.rdhei_side_unpack_job_size.restype = ctypes.c_size_t
assert _lib.rdhei_side_pack_job_size() == ctypes.sizeof(SidePackJob), "rdhei_side_pack_job layout mismatch"
assert _lib.rdhei_side_unpack_job_size() == ctypes.sizeof(SideUnpackJob), "rdhei_side_unpack_job layout mismatch"


def _host_u8(a, nbytes=None):
    import numpy as np
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint8).reshape(-1))
    if nbytes is not None and a.size < nbytes:
        a = np.concatenate([a, np.zeros(nbytes - a.size, np.uint8)])
    return a


_lib.rdhei_b_candidates.argtypes = [ctypes.POINTER(ctypes.c_uint32), ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_uint64)]
_lib.rdhei_b_candidates.restype = ctypes.c_int


def b_candidates(hist, variant: int) -> list[tuple[int, int]]:
    """(b, capacity) pairs in the order of Eq. optimal_b (rdhei_b_candidates)."""
    h = (ctypes.c_uint32 * 9)(*[int(v) for v in hist])
    order, cap = (ctypes.c_int32 * 7)(), (ctypes.c_uint64 * 7)()
    n = _lib.rdhei_b_candidates(h, int(variant), order, cap)
    if n < 0:
        raise RdheiError("rdhei_b_candidates rejected its arguments")
    return [(int(order[k]), int(cap[k])) for k in range(n)]


def bilevel_encode(bits, H: int, W: int) -> bytes:
    """Compress H * W packed bits (host) with the library's bi-level coder."""
    import numpy as np
    src = _host_u8(bits, (H * W + 7) // 8)
    cap = (H * W) // 4 + 64
    out = np.zeros(cap, np.uint8)
    n = ctypes.c_size_t(0)
    _check(_lib.rdhei_bilevel_encode(src.ctypes.data, H, W, out.ctypes.data, cap, ctypes.byref(n)),
           "rdhei_bilevel_encode")
    return out[: n.value].tobytes()


def bilevel_decode(data: bytes, H: int, W: int):
    import numpy as np
    src = np.frombuffer(bytes(data), np.uint8)
    out = np.zeros((H * W + 7) // 8, np.uint8)
    _check(_lib.rdhei_bilevel_decode(src.ctypes.data if src.size else None, src.size, H, W, out.ctypes.data),
           "rdhei_bilevel_decode")
    return out


def lmr_side_pack(items, threads: int = 0) -> list[dict]:
    """items: (eta_bits, map_bits, H, W, b) with host packed maps.  Per item: status,
    the container bytes and its bit length (RDHEI_ECAPACITY when it does not fit)."""
    import numpy as np
    keep, jobs = [], (SidePackJob * len(items))()
    for i, (eta, lm, H, W, b) in enumerate(items):
        nb = (H * W + 7) // 8
        e, m, s = _host_u8(eta, nb), _host_u8(lm, nb), np.zeros(max((H * W) // 8, 1), np.uint8)
        keep.append((e, m, s))
        jobs[i].H, jobs[i].W, jobs[i].b = H, W, b
        jobs[i].eta_bits, jobs[i].map_bits, jobs[i].side = e.ctypes.data, m.ctypes.data, s.ctypes.data
    _check(_lib.rdhei_lmr_side_pack(jobs, len(items), threads), "rdhei_lmr_side_pack")
    out = []
    for i in range(len(items)):
        nbits = int(jobs[i].side_nbits)
        out.append({"status": int(jobs[i].status), "side_nbits": nbits, "side": keep[i][2][: nbits // 8].copy()})
    return out


def lmr_side_unpack(items, threads: int = 0) -> list[dict]:
    """items: (plane, H, W) with the host first-MSB plane.  Per item: status, b and the
    packed rot(eta), rot(l)."""
    import numpy as np
    keep, jobs = [], (SideUnpackJob * len(items))()
    for i, (plane, H, W) in enumerate(items):
        nb = (H * W + 7) // 8
        p, e, m = _host_u8(plane, nb), np.zeros(nb, np.uint8), np.zeros(nb, np.uint8)
        keep.append((p, e, m))
        jobs[i].H, jobs[i].W = H, W
        jobs[i].plane, jobs[i].eta_bits, jobs[i].map_bits = p.ctypes.data, e.ctypes.data, m.ctypes.data
    _check(_lib.rdhei_lmr_side_unpack(jobs, len(items), threads), "rdhei_lmr_side_unpack")
    return [{"status": int(jobs[i].status), "b": int(jobs[i].b), "eta_bits": keep[i][1], "map_bits": keep[i][2]}
            for i in range(len(items))]


def msb_plane(img: torch.Tensor, stream=None) -> torch.Tensor:
    """Bit 7 of every pixel of a device image, packed (device, word-padded)."""
    H, W = img.shape
    out = bitbuf(H * W, img.device)
    _check(_lib.rdhei_msb_plane(_ptr(img), H, W, _ptr(out), _stream(stream)), "rdhei_msb_plane")
    return out
