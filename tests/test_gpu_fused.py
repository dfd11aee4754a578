"""GPU parity of the fused calls through the C ABI.

rdhei_encode (owner + hider) must give, byte for byte, the marked image, maps, label
histogram, b, capacity and embedded count that the oracle's label_encrypt followed by
its embed gives; rdhei_decode (receiver with both keys) the oracle's extracted bits and
recovered image.  Integer path: the bar is bit-exact equality.

Shapes span several 64-row strips and 8192-pixel chunks, ragged tiles and strips, and
rows that do not start on a word of the packed maps; payloads run short, full and past
the capacity so the strips' slot ranges start and end inside 32-bit words.
"""
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


def _fused(rd, img_np, variant, seed, frac=1.0, side_frac=0.3, max_frac=1.0, **kw):
    H, W = img_np.shape
    p, op = _params(rd, variant, seed, **kw)
    nb = (H * W + 7) // 8
    lmr = (variant & 1) == oracle.LMR
    side_n = int(H * W * side_frac) if lmr else 0
    side = synth.random_bits(seed, side_n) if side_n else None
    r = oracle.label_encrypt(op, img_np, side, side_n)
    nbits = int(r.capacity * frac)
    pay = synth.payload_bits(seed, nbits)
    lmr_map_np = r.map_bits if lmr else None
    mref, kref = oracle.embed(op, r.b, r.enc, pay, nbits, lmr_map_np)

    img = torch.from_numpy(img_np).cuda()
    e = rd.encode(img, p, torch.from_numpy(pay).cuda(), nbits,
                  torch.from_numpy(side).cuda() if side_n else None, side_n)
    assert e["hist"] == [int(v) for v in r.hist], "label histogram"
    assert e["b"] == r.b and e["capacity"] == r.capacity, "b / capacity"
    assert e["embedded"] == kref, "embedded bits"
    assert e["status"] == (2 if nbits > r.capacity else 0)
    assert np.array_equal(_np(e["marked"]), mref), "marked image"
    assert np.array_equal(_np(e["map_bits"], nb), r.map_bits), "rotated location map"
    if lmr:
        assert np.array_equal(_np(e["eta_bits"], nb), r.eta_bits), "rotated first-MSB map"

    max_bits = int(r.capacity * max_frac)
    xref, xk = oracle.extract(op, r.b, mref, max_bits, lmr_map_np)
    rref = oracle.decrypt_recover(op, r.b, mref, lmr_map_np, r.eta_bits if lmr else None)
    x = rd.decode(e["marked"], p, r.b, max_bits, e["map_bits"] if lmr else None, e["eta_bits"] if lmr else None)
    assert x["extracted"] == xk
    got = _np(x["bits"])
    assert np.array_equal(got[: (xk + 7) // 8], xref), "extracted bits"
    if xk % 8:
        assert got[xk // 8] & (0xFF >> (xk % 8)) == 0, "padding bits of the last byte"
    assert not got[(xk + 7) // 8:].any(), "zero-filled tail"
    assert np.array_equal(_np(x["recovered"]), rref), "recovered image"
    if lmr:
        assert np.array_equal(rref, img_np)
    return r


SHAPES = [(512, 512), (64, 64), (96, 160), (100, 130), (1, 50), (50, 1), (3, 3), (128, 1024), (200, 72),
          (257, 333), (65, 64), (64, 65), (2, 2), (130, 4100), (700, 96)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("variant", [oracle.EMR, oracle.LMR])
def test_fused_shapes(rd, shape, variant):
    H, W = shape
    seed = H * 1000 + W + variant + 77
    _fused(rd, synth.synth_image(H, W, seed), variant, seed)


@pytest.mark.parametrize("variant", [oracle.EMR, oracle.LMR, oracle.EMR_MED, oracle.LMR_MED])
@pytest.mark.parametrize("kw", [dict(rot_enable=0), dict(rot_lmin=2), dict(rot_lmin=3), dict(rot_lmin=4), dict(b=3),
                                dict(b=6)])
def test_fused_parameters(rd, variant, kw):
    img = synth.synth_image(256, 320, 5, noise_sigma=2.0)
    _fused(rd, img, variant, 19, **kw)


@pytest.mark.parametrize("frac,max_frac", [(0.0, 1.0), (0.013, 1.0), (0.5, 0.5), (1.0, 0.37), (1.6, 1.0),
                                           (1.0, 2.0)])
def test_fused_partial_payload_and_limits(rd, frac, max_frac):
    img = synth.synth_image(320, 448, 9)
    _fused(rd, img, oracle.EMR, 29, frac=frac, max_frac=max_frac)
    _fused(rd, img, oracle.LMR, 30, frac=frac, max_frac=max_frac)


@pytest.mark.parametrize("shape,frac", [((150, 1040), 1.0), ((150, 1040), 0.41), ((64, 2048), 0.2),
                                        ((64, 2048), 1.0), ((97, 528), 0.77), ((70, 16), 1.0)])
def test_fused_wide_rows_and_short_messages(rd, shape, frac):
    """Rows of several 512-pixel spans, strips whose message ends mid-row or overflows
    one staged window of K2 words, and an image narrower than a 16-pixel load."""
    H, W = shape
    img = synth.synth_image(H, W, H + W)
    _fused(rd, img, oracle.EMR, 40 + H, frac=frac)
    _fused(rd, img, oracle.LMR, 41 + H, frac=frac)


def test_fused_edge_images(rd):
    # constant (every non-first pixel redundant, b = 7), no redundancy at all (no slots),
    # and an image whose top half has no slots (whole strips with empty slot ranges)
    _fused(rd, np.full((130, 200), 91, np.uint8), oracle.EMR, 31)
    _fused(rd, np.full((130, 200), 91, np.uint8), oracle.LMR, 31)
    stripes = np.tile(np.array([0, 255], np.uint8), (70, 90))
    _fused(rd, stripes, oracle.EMR, 32)
    half = synth.synth_image(256, 200, 33, noise_sigma=1.0)
    half[:128] = np.tile(np.array([0, 255], np.uint8), (128, 100))
    _fused(rd, half, oracle.EMR, 33)
    _fused(rd, half, oracle.LMR, 34)
    noise = np.random.default_rng(3).integers(0, 256, size=(300, 300)).astype(np.uint8)
    _fused(rd, noise, oracle.EMR, 35)


def test_fused_equals_separable_batch(rd):
    """A mixed batch of uneven sizes and all four variants in one plan per fused call;
    every image equals the separable four-call chain run on the same batch."""
    rng = np.random.default_rng(41)
    shapes = [(512, 512), (256, 1024), (333, 257), (64, 4096), (1000, 72), (129, 130), (40, 40), (512, 96)]
    imgs = [synth.synth_image(h, w, 500 + i, noise_sigma=float(rng.uniform(1, 16))) for i, (h, w) in enumerate(shapes)]
    variants = [[oracle.EMR, oracle.LMR, oracle.EMR_MED, oracle.LMR_MED][i % 4] for i in range(len(imgs))]
    n = len(imgs)
    P = []
    for i in range(n):
        k = synth.keys(600 + i)
        P.append(rd.Params(variant=variants[i], k1=k["k1"], nonce1=k["nonce1"], k2=k["k2"], nonce2=k["nonce2"]))
    d_img = [torch.from_numpy(im).cuda() for im in imgs]
    N = [im.size for im in imgs]
    lmr = [(v & 1) == rd.LMR for v in variants]
    side_n = [N[i] // 5 if lmr[i] else 0 for i in range(n)]
    sides = [rd.as_bitbuf(torch.from_numpy(synth.random_bits(700 + i, side_n[i])), side_n[i]) if side_n[i] else None
             for i in range(n)]

    # separable chain
    info_a = rd.new_info(n)
    enc = [torch.empty_like(x) for x in d_img]
    maps_a = [rd.bitbuf(N[i]) for i in range(n)]
    etas_a = [rd.bitbuf(N[i]) for i in range(n)]
    rd.Plan([rd.make_job(P[i], *imgs[i].shape, src=d_img[i], dst=enc[i], map_bits=maps_a[i],
                         eta_bits=etas_a[i] if lmr[i] else None, side_bits=sides[i], side_nbits=side_n[i],
                         info=info_a[i]) for i in range(n)]).run(rd.OP_LABEL_ENCRYPT)
    torch.cuda.synchronize()
    caps = [r["capacity"] for r in rd.read_info(info_a)]
    pays = [rd.as_bitbuf(torch.from_numpy(synth.payload_bits(800 + i, caps[i])), caps[i]) for i in range(n)]
    marked_a = [torch.empty_like(x) for x in d_img]
    rd.Plan([rd.make_job(P[i], *imgs[i].shape, src=enc[i], dst=marked_a[i], map_bits=maps_a[i] if lmr[i] else None,
                         payload=pays[i], nbits=caps[i], info=info_a[i], b=0) for i in range(n)]).run(rd.OP_EMBED)
    bits_a = [rd.bitbuf(caps[i]) for i in range(n)]
    rec_a = [torch.empty_like(x) for x in d_img]
    rd.Plan([rd.make_job(P[i], *imgs[i].shape, src=marked_a[i], map_bits=maps_a[i] if lmr[i] else None,
                         bits_out=bits_a[i], max_bits=caps[i], info=info_a[i], b=0) for i in range(n)]).run(rd.OP_EXTRACT)
    rd.Plan([rd.make_job(P[i], *imgs[i].shape, src=marked_a[i], dst=rec_a[i], map_bits=maps_a[i] if lmr[i] else None,
                         eta_bits=etas_a[i] if lmr[i] else None, info=info_a[i], b=0) for i in range(n)]
            ).run(rd.OP_DECRYPT_RECOVER)

    # fused calls, one plan each
    info_b = rd.new_info(n)
    marked_b = [torch.empty_like(x) for x in d_img]
    maps_b = [rd.bitbuf(N[i]) for i in range(n)]
    etas_b = [rd.bitbuf(N[i]) for i in range(n)]
    pe = rd.Plan([rd.make_job(P[i], *imgs[i].shape, src=d_img[i], dst=marked_b[i], map_bits=maps_b[i],
                              eta_bits=etas_b[i] if lmr[i] else None, side_bits=sides[i], side_nbits=side_n[i],
                              payload=pays[i], nbits=caps[i], info=info_b[i]) for i in range(n)])
    pe.run(rd.OP_ENCODE)
    bits_b = [rd.bitbuf(caps[i]) for i in range(n)]
    rec_b = [torch.empty_like(x) for x in d_img]
    pd = rd.Plan([rd.make_job(P[i], *imgs[i].shape, src=marked_b[i], dst=rec_b[i],
                              map_bits=maps_b[i] if lmr[i] else None, eta_bits=etas_b[i] if lmr[i] else None,
                              bits_out=bits_b[i], max_bits=caps[i], info=info_b[i], b=0) for i in range(n)])
    pd.run(rd.OP_DECODE)
    torch.cuda.synchronize()
    assert pe.status() == 0 and pd.status() == 0
    ia, ib = rd.read_info(info_a), rd.read_info(info_b)
    for i in range(n):
        assert ia[i]["b"] == ib[i]["b"] and ia[i]["capacity"] == ib[i]["capacity"], i
        assert ib[i]["embedded"] == caps[i] and ib[i]["extracted"] == caps[i], i
        assert torch.equal(marked_a[i], marked_b[i]), f"marked image {i}"
        assert torch.equal(maps_a[i], maps_b[i]), f"map {i}"
        assert torch.equal(bits_a[i], bits_b[i]), f"bits {i}"
        assert torch.equal(bits_b[i][: (caps[i] + 7) // 8].cpu(), pays[i][: (caps[i] + 7) // 8].cpu()), f"payload {i}"
        assert torch.equal(rec_a[i], rec_b[i]), f"recovered {i}"
        if lmr[i] and variants[i] < 2:
            assert torch.equal(rec_b[i].cpu(), torch.from_numpy(imgs[i])), f"lossless {i}"

    # the plans rerun (captured-graph style reuse) and give the same bytes
    pe.run(rd.OP_ENCODE)
    pd.run(rd.OP_DECODE)
    torch.cuda.synchronize()
    for i in range(n):
        assert torch.equal(marked_a[i], marked_b[i]) and torch.equal(bits_a[i], bits_b[i])
        assert torch.equal(rec_a[i], rec_b[i])


def test_fused_rejects_missing_buffers(rd):
    p, _ = _params(rd, rd.LMR, 3)
    img = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(img)
    info = rd.new_info(1)
    # LMR encode without map_bits: the hider's half needs the rotated map
    j = rd.make_job(p, 64, 64, src=img, dst=out, info=info)
    with pytest.raises(rd.RdheiError):
        rd.run_jobs(rd.OP_ENCODE, [j])
    # decode without its output image
    j = rd.make_job(p, 64, 64, src=img, map_bits=rd.bitbuf(4096), eta_bits=rd.bitbuf(4096), info=info)
    with pytest.raises(rd.RdheiError):
        rd.run_jobs(rd.OP_DECODE, [j])


def test_async_upload_on_a_side_stream(rd):
    """Plans whose descriptors go up from a pinned staging buffer (rdhei_plan_upload_async),
    created and run on a non-default stream with no synchronisation in between, give the
    bytes of plans uploaded synchronously; a staging buffer that is missing or too small
    is refused before anything is queued."""
    shapes = [(300, 470), (64, 4096), (129, 130)]
    variants = [oracle.EMR, oracle.LMR, oracle.LMR_MED]
    n = len(shapes)
    imgs = [torch.from_numpy(synth.synth_image(h, w, 900 + i)).cuda() for i, (h, w) in enumerate(shapes)]
    P = [_params(rd, variants[i], 910 + i)[0] for i in range(n)]
    lmr = [(v & 1) == rd.LMR for v in variants]
    caps = [im.numel() for im in imgs]          # payload longer than any capacity: embedding stops there
    pays = [rd.as_bitbuf(torch.from_numpy(synth.payload_bits(920 + i, caps[i])), caps[i]) for i in range(n)]

    def run(staged, stream):
        info = rd.new_info(n)
        marked = [torch.empty_like(x) for x in imgs]
        maps = [rd.bitbuf(x.numel()) for x in imgs]
        etas = [rd.bitbuf(x.numel()) if lmr[i] else None for i, x in enumerate(imgs)]
        bits = [rd.bitbuf(caps[i]) for i in range(n)]
        rec = [torch.empty_like(x) for x in imgs]
        stage = (lambda nb: torch.empty(nb, dtype=torch.uint8, pin_memory=True)) if staged else None
        with torch.cuda.stream(stream):
            pe = rd.Plan([rd.make_job(P[i], *shapes[i], src=imgs[i], dst=marked[i], map_bits=maps[i],
                                      eta_bits=etas[i], payload=pays[i], nbits=caps[i], info=info[i])
                          for i in range(n)], stream, staging=stage)
            pe.run(rd.OP_ENCODE, stream)
            pd = rd.Plan([rd.make_job(P[i], *shapes[i], src=marked[i], dst=rec[i],
                                      map_bits=maps[i] if lmr[i] else None, eta_bits=etas[i], bits_out=bits[i],
                                      max_bits=caps[i], info=info[i], b=0) for i in range(n)], stream, staging=stage)
            pd.run(rd.OP_DECODE, stream)
        stream.synchronize()
        assert pe.status() in (0, rd.RDHEI_ECAPACITY) and pd.status() == 0
        return [t.cpu() for t in marked + bits + rec], rd.read_info(info)

    torch.cuda.synchronize()
    ref, iref = run(False, torch.cuda.current_stream())
    got, igot = run(True, torch.cuda.Stream())
    assert iref == igot
    for a, b in zip(ref, got):
        assert torch.equal(a, b)

    plan = rd.Plan([rd.make_job(P[0], *shapes[0], src=imgs[0], dst=torch.empty_like(imgs[0]), info=rd.new_info(1))])
    need = int(rd._lib.rdhei_plan_staging_size(plan._h))
    small = torch.empty(max(need - 16, 16), dtype=torch.uint8, pin_memory=True)
    import ctypes
    rc = rd._lib.rdhei_plan_upload_async(plan._h, ctypes.c_void_p(plan._ws_ptr), plan._ws_bytes,
                                         ctypes.c_void_p(small.data_ptr()), small.numel(), None)
    assert rc == rd.RDHEI_ESPACE
    rc = rd._lib.rdhei_plan_upload_async(plan._h, ctypes.c_void_p(plan._ws_ptr), plan._ws_bytes, None, 0, None)
    assert rc == rd.RDHEI_EINVAL
