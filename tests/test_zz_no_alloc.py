"""rdhei_extract_noalloc: extraction for callers that cannot allocate device memory
(it runs on a static device array instead of a caller-provided workspace).  Its
output must equal rdhei_extract's, call after call, since every call reuses -- and
clears -- the same array.  This file is collected last on purpose."""
import numpy as np
import pytest
import torch

from paper_2302_07992_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rd():
    from paper_2302_07992_gb300 import rdhei
    return rdhei


def _prepared(rd, variant, H, W, seed):
    k = synth.keys(seed)
    p = rd.Params(variant=variant, k1=k["k1"], nonce1=k["nonce1"], k2=k["k2"], nonce2=k["nonce2"])
    img = torch.from_numpy(synth.synth_image(H, W, seed)).cuda()
    e = rd.label_encrypt(img, p)
    nbits = e["capacity"]
    pay = torch.from_numpy(synth.payload_bits(seed, nbits)).cuda()
    lmap = e["map_bits"] if variant == rd.LMR else None
    m = rd.embed(e["enc"], p, e["b"], pay, nbits, lmap)
    return p, e, m["marked"], lmap, nbits, pay


@pytest.mark.parametrize("variant,shape,frac", [(0, (512, 512), 1.0), (1, (300, 470), 1.0), (0, (97, 1000), 0.37),
                                               (1, (64, 65), 0.5)])
def test_noalloc_matches_extract_twice(rd, variant, shape, frac):
    H, W = shape
    p, e, marked, lmap, cap, pay = _prepared(rd, variant, H, W, 7000 + H + variant)
    max_bits = int(cap * frac)
    ref = rd.extract(marked, p, e["b"], max_bits, lmap)
    nb = (ref["extracted"] + 7) // 8
    for _ in range(2):                                   # the shared array keeps the last call's contents
        out = rd.bitbuf(max_bits)
        out.fill_(0xA5)                                  # stale bytes must not leak into the result
        info = rd.new_info(1)
        job = rd.make_job(p, H, W, src=marked, map_bits=lmap, bits_out=out, max_bits=max_bits, info=info,
                          b=e["b"])
        assert rd.extract_noalloc_job(job) == 0
        torch.cuda.synchronize()
        got = rd.read_info(info)[0]
        assert got["extracted"] == ref["extracted"]
        assert torch.equal(out[:nb], ref["bits"][:nb])
        full = ref["extracted"] // 8
        assert torch.equal(out[:full], pay[:full])       # and it is the embedded payload


def test_noalloc_rejects_images_beyond_its_array(rd):
    p = rd.Params()
    info = rd.new_info(1)
    dummy = torch.zeros(16, dtype=torch.uint8, device="cuda")
    job = rd.make_job(p, 4097, 4097, src=dummy, bits_out=dummy, max_bits=8, info=info)
    assert rd.extract_noalloc_job(job) == 5            # RDHEI_ESPACE, before any GPU work
