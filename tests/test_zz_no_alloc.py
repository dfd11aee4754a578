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
        assert got["extracted"] == ref["extracted"] and got["status"] == 0
        assert torch.equal(out[:nb], ref["bits"][:nb])
        full = ref["extracted"] // 8
        assert torch.equal(out[:full], pay[:full])       # and it is the embedded payload


def test_noalloc_rejects_images_beyond_its_array(rd):
    p = rd.Params()
    info = rd.new_info(1)
    dummy = torch.zeros(16, dtype=torch.uint8, device="cuda")
    job = rd.make_job(p, 4097, 4097, src=dummy, bits_out=dummy, max_bits=8, info=info)
    assert rd.extract_noalloc_job(job) == 5            # RDHEI_ESPACE, before any GPU work


def _noalloc(rd, p, H, W, marked, lmap, max_bits, b, stream=None, fill=0xA5):
    out = rd.bitbuf(max_bits)
    out.fill_(fill)
    info = rd.new_info(1)
    job = rd.make_job(p, H, W, src=marked, map_bits=lmap, bits_out=out, max_bits=max_bits, info=info, b=b)
    assert rd.extract_noalloc_job(job, stream) == 0
    return out, info


@pytest.mark.parametrize("variant", [0, 1])
def test_noalloc_largest_image(rd, variant):
    """H * W = 2^24 fills the array's chunk table exactly."""
    H = W = 4096
    p, e, marked, lmap, cap, pay = _prepared(rd, variant, H, W, 7100 + variant)
    ref = rd.extract(marked, p, e["b"], cap, lmap)
    out, info = _noalloc(rd, p, H, W, marked, lmap, cap, e["b"])
    torch.cuda.synchronize()
    got = rd.read_info(info)[0]
    nb = (ref["extracted"] + 7) // 8
    assert got["extracted"] == ref["extracted"] == cap and got["status"] == 0
    assert torch.equal(out[:nb], ref["bits"][:nb])


def test_noalloc_large_then_small_on_a_side_stream(rd):
    """A large call followed by a smaller one on a non-default stream: the counts and
    offsets the large call left in the array must not leak into the small one."""
    s = torch.cuda.Stream()
    big = _prepared(rd, 0, 1500, 1700, 7201)
    small = _prepared(rd, 1, 130, 210, 7202)
    refs = []
    for (p, e, marked, lmap, cap, pay), (H, W) in ((big, (1500, 1700)), (small, (130, 210))):
        refs.append(rd.extract(marked, p, e["b"], cap, lmap))
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        outs = []
        for (p, e, marked, lmap, cap, pay), (H, W) in ((big, (1500, 1700)), (small, (130, 210)),
                                                       (big, (1500, 1700))):
            outs.append(_noalloc(rd, p, H, W, marked, lmap, cap, e["b"], stream=s))
    s.synchronize()
    for (out, info), ref in zip(outs, refs + refs[:1]):
        got = rd.read_info(info)[0]
        nb = (ref["extracted"] + 7) // 8
        assert got["extracted"] == ref["extracted"] and got["status"] == 0
        assert torch.equal(out[:nb], ref["bits"][:nb])


def test_noalloc_refuses_a_capturing_stream(rd):
    """Each call uploads its descriptor from a host stack buffer, so a call on a stream
    that is being captured returns RDHEI_EINVAL and enqueues nothing."""
    p, e, marked, lmap, cap, pay = _prepared(rd, 0, 96, 128, 7301)
    out = rd.bitbuf(cap)
    info = rd.new_info(1)
    job = rd.make_job(p, 96, 128, src=marked, bits_out=out, max_bits=cap, info=info, b=e["b"])
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            rc = rd.extract_noalloc_job(job, s)
        finally:
            g.capture_end()
    assert rc == 1                                      # RDHEI_EINVAL
    # the stream and the array still work afterwards
    out2, info2 = _noalloc(rd, p, 96, 128, marked, None, cap, e["b"])
    torch.cuda.synchronize()
    ref = rd.extract(marked, p, e["b"], cap)
    nb = (cap + 7) // 8
    assert torch.equal(out2[:nb], ref["bits"][:nb])
