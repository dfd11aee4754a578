"""GPU parity on the workload shapes of the benchmark configurations, through the
batched (plan) path: many images of uneven sizes and both variants in one launch per
operation, each image's outputs equal to the CPU oracle's byte for byte.

  * 512 x 512 batch with per-image smoothness, EMR and LMR mixed;
  * uneven sizes drawn from {256, ..., 4096} per axis plus ragged sides;
  * the largest size, 8192 x 8192;
  * decode-only on 4096 x 4096 images marked by the oracle (GPU receivers on inputs the
    GPU did not produce).
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


def _keys(seed):
    k = synth.keys(seed)
    return dict(k1=k["k1"], nonce1=k["nonce1"], k2=k["k2"], nonce2=k["nonce2"])


def _bits(t, n):
    return t.detach().cpu().numpy()[: (n + 7) // 8]


def _packed(imgs, fill=None, skew=0):
    """Images laid end to end in one flat device buffer, each starting at an odd byte
    offset (no 16-, 4- or 2-byte alignment)."""
    sizes = [im.size for im in imgs]
    flat = torch.zeros(sum(sizes) + 8 * len(imgs) + 16, dtype=torch.uint8, device="cuda")
    out, off = [], 1 + skew
    for im in imgs:
        v = flat[off: off + im.size].view(*im.shape)
        if fill is not None:
            v.copy_(torch.from_numpy(np.ascontiguousarray(im)))
        out.append(v)
        off += im.size + 3 + 2 * (off % 3)
    return out


def _run_batch(rd, imgs, variants, seeds, side_frac=0.125, odd_offsets=False):
    """All four operations, one plan (one launch sequence) per operation."""
    n = len(imgs)
    P = [rd.Params(variant=v, **_keys(s)) for v, s in zip(variants, seeds)]
    if odd_offsets:
        d_img = _packed(imgs, fill=True)
        enc, marked, rec = _packed(imgs, skew=2), _packed(imgs, skew=4), _packed(imgs, skew=6)
    else:
        d_img = [torch.from_numpy(np.ascontiguousarray(im)).cuda() for im in imgs]
        enc = [torch.empty_like(x) for x in d_img]
        marked = [torch.empty_like(x) for x in d_img]
        rec = [torch.empty_like(x) for x in d_img]
    N = [im.size for im in imgs]
    maps = [rd.bitbuf(N[i]) for i in range(n)]
    etas = [rd.bitbuf(N[i]) for i in range(n)]
    side_n = [int(N[i] * side_frac) if variants[i] == rd.LMR else 0 for i in range(n)]
    side_np = [synth.random_bits(seeds[i], side_n[i]) if side_n[i] else None for i in range(n)]
    sides = [rd.as_bitbuf(torch.from_numpy(side_np[i]), side_n[i]) if side_n[i] else None for i in range(n)]
    info = rd.new_info(n)
    jobs = [rd.make_job(P[i], *imgs[i].shape, src=d_img[i], dst=enc[i], map_bits=maps[i],
                        eta_bits=etas[i] if variants[i] == rd.LMR else None, side_bits=sides[i], side_nbits=side_n[i],
                        info=info[i]) for i in range(n)]
    rd.Plan(jobs).run(rd.OP_LABEL_ENCRYPT)
    torch.cuda.synchronize()
    inf = rd.read_info(info)
    caps = [r["capacity"] for r in inf]
    pays = [synth.payload_bits(seeds[i], caps[i]) for i in range(n)]
    d_pay = [rd.as_bitbuf(torch.from_numpy(pays[i]), caps[i]) for i in range(n)]
    bits = [rd.bitbuf(caps[i]) for i in range(n)]
    lm = [maps[i] if variants[i] == rd.LMR else None for i in range(n)]
    rd.Plan([rd.make_job(P[i], *imgs[i].shape, src=enc[i], dst=marked[i], map_bits=lm[i], payload=d_pay[i],
                         nbits=caps[i], info=info[i], b=0) for i in range(n)]).run(rd.OP_EMBED)
    rd.Plan([rd.make_job(P[i], *imgs[i].shape, src=marked[i], map_bits=lm[i], bits_out=bits[i], max_bits=caps[i],
                         info=info[i], b=0) for i in range(n)]).run(rd.OP_EXTRACT)
    rd.Plan([rd.make_job(P[i], *imgs[i].shape, src=marked[i], dst=rec[i], map_bits=lm[i],
                         eta_bits=etas[i] if variants[i] == rd.LMR else None, info=info[i], b=0)
             for i in range(n)]).run(rd.OP_DECRYPT_RECOVER)
    torch.cuda.synchronize()
    return dict(P=P, enc=enc, marked=marked, rec=rec, maps=maps, etas=etas, bits=bits, info=rd.read_info(info),
                caps=caps, pays=pays, side_np=side_np, side_n=side_n)


def _check_against_oracle(rd, imgs, variants, seeds, out, i):
    img, v = imgs[i], variants[i]
    op = oracle.Params(variant=v, **_keys(seeds[i]))
    H, W = img.shape
    r = oracle.label_encrypt(op, img, out["side_np"][i], out["side_n"][i])
    g = out["info"][i]
    assert g["hist"] == [int(x) for x in r.hist] and g["b"] == r.b and g["capacity"] == r.capacity, i
    assert np.array_equal(out["enc"][i].cpu().numpy(), r.enc), i
    assert np.array_equal(_bits(out["maps"][i], H * W), r.map_bits), i
    lm = r.map_bits if v == oracle.LMR else None
    mref, k = oracle.embed(op, r.b, r.enc, out["pays"][i], r.capacity, lm)
    assert np.array_equal(out["marked"][i].cpu().numpy(), mref), i
    xref, xk = oracle.extract(op, r.b, mref, r.capacity, lm)
    assert g["extracted"] == xk and np.array_equal(_bits(out["bits"][i], xk), xref), i
    rref = oracle.decrypt_recover(op, r.b, mref, lm, r.eta_bits if v == oracle.LMR else None)
    assert np.array_equal(out["rec"][i].cpu().numpy(), rref), i


def test_batch_512_mixed_variants(rd):
    n = 24
    imgs = [synth.batch_image(2, k, 512, 512, vary=True) for k in range(n)]
    variants = [rd.EMR if k % 2 == 0 else rd.LMR for k in range(n)]
    seeds = [synth.image_seed(2, k) for k in range(n)]
    out = _run_batch(rd, imgs, variants, seeds)
    for i in range(n):
        _check_against_oracle(rd, imgs, variants, seeds, out, i)


def test_uneven_sizes_one_launch(rd):
    rng = np.random.default_rng(33)
    sides = [256, 512, 1024, 2048]
    shapes = [(int(rng.choice(sides)), int(rng.choice(sides))) for _ in range(8)]
    shapes += [(4096, 256), (1000, 777), (333, 2048), (4096, 4096)]
    imgs = [synth.synth_image(H, W, 100 + i) for i, (H, W) in enumerate(shapes)]
    variants = [rd.EMR if i % 3 else rd.LMR for i in range(len(shapes))]
    seeds = [500 + i for i in range(len(shapes))]
    out = _run_batch(rd, imgs, variants, seeds)
    for i in range(len(shapes)):
        _check_against_oracle(rd, imgs, variants, seeds, out, i)


def test_images_at_odd_byte_offsets(rd):
    """Source, encrypted, marked and recovered images at odd byte offsets of shared
    buffers, ragged sizes: every kernel's unaligned path against the oracle."""
    shapes = [(100, 130), (257, 333), (64, 64), (1, 50), (333, 1000), (512, 512), (77, 8200)]
    imgs = [synth.synth_image(H, W, 700 + i) for i, (H, W) in enumerate(shapes)]
    variants = [rd.EMR if i % 2 == 0 else rd.LMR for i in range(len(shapes))]
    seeds = [700 + i for i in range(len(shapes))]
    out = _run_batch(rd, imgs, variants, seeds, odd_offsets=True)
    ptrs = [out[k][i].data_ptr() for k in ("enc", "marked", "rec") for i in range(len(shapes))]
    assert sum(p % 16 != 0 for p in ptrs) > len(ptrs) // 2
    for i in range(len(shapes)):
        _check_against_oracle(rd, imgs, variants, seeds, out, i)


@pytest.mark.slow
def test_largest_size_8192(rd):
    """8192 x 8192 (13 rotation levels, 16,384 tiles, 8,192 chunks), EMR, full parity."""
    img = synth.synth_image(8192, 8192, 81)
    out = _run_batch(rd, [img], [rd.EMR], [81])
    _check_against_oracle(rd, [img], [rd.EMR], [81], out, 0)


def test_decode_only_on_oracle_marked_4096(rd):
    """The GPU receivers on 4096 x 4096 images that the oracle encoded and marked."""
    n = 2
    for i in range(n):
        img = synth.synth_image(4096, 4096, 900 + i)
        v = oracle.EMR if i == 0 else oracle.LMR
        op = oracle.Params(variant=v, **_keys(900 + i))
        r = oracle.label_encrypt(op, img)
        pay = synth.payload_bits(900 + i, r.capacity)
        lm = r.map_bits if v == oracle.LMR else None
        mref, _ = oracle.embed(op, r.b, r.enc, pay, r.capacity, lm)
        p = rd.Params(variant=v, **_keys(900 + i))
        dm = torch.from_numpy(mref).cuda()
        dmap = rd.as_bitbuf(torch.from_numpy(r.map_bits), img.size) if lm is not None else None
        deta = rd.as_bitbuf(torch.from_numpy(r.eta_bits), img.size) if lm is not None else None
        x = rd.extract(dm, p, r.b, r.capacity, dmap)
        xref, xk = oracle.extract(op, r.b, mref, r.capacity, lm)
        assert x["extracted"] == xk and np.array_equal(_bits(x["bits"], xk), xref)
        rec = rd.decrypt_recover(dm, p, r.b, dmap, deta)
        rref = oracle.decrypt_recover(op, r.b, mref, lm, r.eta_bits if lm is not None else None)
        assert np.array_equal(rec.cpu().numpy(), rref)


@pytest.mark.parametrize("fused", [False, True])
def test_overlapped_host_pipeline_matches_the_oracle(fused):
    """Host-to-host runs with copies overlapped across chunks give each image's oracle
    result, run after run (buffer reuse between runs is ordered by events), through the
    four separable calls or the two fused ones."""
    import torch
    from paper_2302_07992_gb300 import pipeline as pp
    from paper_2302_07992_gb300 import rdhei as rd
    n, H, W = 10, 96, 160
    variants = [rd.EMR, rd.LMR, rd.EMR_MED, rd.LMR_MED, rd.EMR] * 2
    imgs = np.stack([synth.synth_image(H, W, 700 + k) for k in range(n)])
    params, oparams, caps, refs, pays, sides = [], [], [], [], [], []
    sn = (H * W + 7) // 8
    for k in range(n):
        kk = synth.keys(700 + k)
        common = dict(variant=variants[k], k1=kk["k1"], nonce1=kk["nonce1"], k2=kk["k2"], nonce2=kk["nonce2"])
        params.append(rd.Params(**common))
        oparams.append(oracle.Params(**common))
        lmr = (variants[k] & 1) == rd.LMR
        side = synth.random_bits(700 + k, sn) if lmr else None
        r = oracle.label_encrypt(oparams[k], imgs[k], side, sn if lmr else 0)
        pay = synth.payload_bits(700 + k, r.capacity)
        lm = r.map_bits if lmr else None
        marked, _ = oracle.embed(oparams[k], r.b, r.enc, pay, r.capacity, lm)
        refs.append(oracle.decrypt_recover(oparams[k], r.b, marked, lm, r.eta_bits if lmr else None))
        caps.append(r.capacity)
        pays.append(pay)
        sides.append(side if lmr else np.zeros(1, np.uint8))
    op = pp.OverlappedPipeline(n, H, W, variants, params, caps,
                               side_nbits=[sn if (v & 1) == rd.LMR else 0 for v in variants], chunks=3, fused=fused)
    h_img, h_pay, h_side, h_rec, h_bits = op.host_buffers()
    h_img.copy_(torch.from_numpy(imgs))
    op.pack_payloads(h_pay, pays)
    op.pack_side(h_side, sides)
    for _ in range(3):
        h_rec.zero_()
        h_bits.zero_()
        op.run(h_img, h_pay, h_side, h_rec, h_bits).synchronize()
        torch.cuda.synchronize()
        for k in range(n):
            assert np.array_equal(h_rec[k].numpy(), refs[k]), k
            nb = (caps[k] + 7) // 8
            o = op.pay_off[k]
            assert np.array_equal(h_bits[o:o + nb].numpy(), pays[k][:nb]), k
    assert op.status() == 0


def test_repeated_steps_without_host_synchronisation(rd):
    """Three full steps (label_encrypt, embed, extract, decrypt_recover) queued back to
    back on one stream over the same buffers, with no host synchronisation in between:
    the kernels of an operation and of consecutive operations overlap programmatically,
    and every read-after-write and write-after-read across them must still hold.  The
    final outputs equal the oracle's."""
    shapes = [(512, 512), (100, 130), (257, 333), (64, 1000)]
    variants = [rd.EMR, rd.LMR, rd.EMR_MED, rd.LMR]
    imgs = [synth.synth_image(H, W, 900 + i) for i, (H, W) in enumerate(shapes)]
    seeds = [900 + i for i in range(len(shapes))]
    n = len(imgs)
    P = [rd.Params(variant=v, **_keys(s)) for v, s in zip(variants, seeds)]
    d_img = [torch.from_numpy(np.ascontiguousarray(im)).cuda() for im in imgs]
    enc = [torch.empty_like(x) for x in d_img]
    marked = [torch.empty_like(x) for x in d_img]
    rec = [torch.empty_like(x) for x in d_img]
    N = [im.size for im in imgs]
    lmr = [(v & 1) == rd.LMR for v in variants]
    maps = [rd.bitbuf(N[i]) for i in range(n)]
    etas = [rd.bitbuf(N[i]) for i in range(n)]
    info = rd.new_info(n)
    st = torch.cuda.current_stream()
    p_enc = rd.Plan([rd.make_job(P[i], *imgs[i].shape, src=d_img[i], dst=enc[i], map_bits=maps[i],
                                 eta_bits=etas[i] if lmr[i] else None, info=info[i]) for i in range(n)], st)
    p_enc.run(rd.OP_LABEL_ENCRYPT, st)
    torch.cuda.synchronize()
    caps = [r["capacity"] for r in rd.read_info(info)]
    pays = [synth.payload_bits(seeds[i], caps[i]) for i in range(n)]
    d_pay = [rd.as_bitbuf(torch.from_numpy(pays[i]), caps[i]) for i in range(n)]
    bits = [rd.bitbuf(caps[i]) for i in range(n)]
    lm = [maps[i] if lmr[i] else None for i in range(n)]
    p_emb = rd.Plan([rd.make_job(P[i], *imgs[i].shape, src=enc[i], dst=marked[i], map_bits=lm[i], payload=d_pay[i],
                                 nbits=caps[i], info=info[i], b=0) for i in range(n)], st)
    p_ext = rd.Plan([rd.make_job(P[i], *imgs[i].shape, src=marked[i], map_bits=lm[i], bits_out=bits[i],
                                 max_bits=caps[i], info=info[i], b=0) for i in range(n)], st)
    p_dec = rd.Plan([rd.make_job(P[i], *imgs[i].shape, src=marked[i], dst=rec[i], map_bits=lm[i],
                                 eta_bits=etas[i] if lmr[i] else None, info=info[i], b=0) for i in range(n)], st)
    torch.cuda.synchronize()
    for _ in range(3):
        for pl, op in ((p_enc, rd.OP_LABEL_ENCRYPT), (p_emb, rd.OP_EMBED), (p_ext, rd.OP_EXTRACT),
                       (p_dec, rd.OP_DECRYPT_RECOVER)):
            pl.run(op, st)
    torch.cuda.synchronize()
    for pl in (p_enc, p_emb, p_ext, p_dec):
        assert pl.status(st) == 0
    for i in range(n):
        op = oracle.Params(variant=variants[i], **_keys(seeds[i]))
        r = oracle.label_encrypt(op, imgs[i])
        assert np.array_equal(enc[i].cpu().numpy(), r.enc), i
        l_np = r.map_bits if lmr[i] else None
        mref, _ = oracle.embed(op, r.b, r.enc, pays[i], r.capacity, l_np)
        assert np.array_equal(marked[i].cpu().numpy(), mref), i
        xref, xk = oracle.extract(op, r.b, mref, r.capacity, l_np)
        assert np.array_equal(_bits(bits[i], xk), xref), i
        rref = oracle.decrypt_recover(op, r.b, mref, l_np, r.eta_bits if lmr[i] else None)
        assert np.array_equal(rec[i].cpu().numpy(), rref), i



def test_repeated_fused_steps_without_host_synchronisation(rd):
    """The fused calls queued back to back three times over the same buffers with no host
    synchronisation: the final outputs equal the oracle's."""
    shapes = [(512, 512), (100, 130), (257, 333), (64, 1000), (700, 96)]
    variants = [rd.EMR, rd.LMR, rd.EMR_MED, rd.LMR, rd.LMR_MED]
    imgs = [synth.synth_image(H, W, 950 + i) for i, (H, W) in enumerate(shapes)]
    seeds = [950 + i for i in range(len(shapes))]
    n = len(imgs)
    P = [rd.Params(variant=v, **_keys(s)) for v, s in zip(variants, seeds)]
    d_img = [torch.from_numpy(np.ascontiguousarray(im)).cuda() for im in imgs]
    scratch = [torch.empty_like(x) for x in d_img]
    marked = [torch.empty_like(x) for x in d_img]
    rec = [torch.empty_like(x) for x in d_img]
    N = [im.size for im in imgs]
    lmr = [(v & 1) == rd.LMR for v in variants]
    maps = [rd.bitbuf(N[i]) for i in range(n)]
    etas = [rd.bitbuf(N[i]) for i in range(n)]
    info = rd.new_info(n)
    st = torch.cuda.current_stream()
    rd.Plan([rd.make_job(P[i], *imgs[i].shape, src=d_img[i], dst=scratch[i], info=info[i]) for i in range(n)],
            st).run(rd.OP_LABEL_ENCRYPT, st)
    torch.cuda.synchronize()
    caps = [r["capacity"] for r in rd.read_info(info)]
    pays = [synth.payload_bits(seeds[i], caps[i]) for i in range(n)]
    d_pay = [rd.as_bitbuf(torch.from_numpy(pays[i]), caps[i]) for i in range(n)]
    bits = [rd.bitbuf(caps[i]) for i in range(n)]
    lm = [maps[i] if lmr[i] else None for i in range(n)]
    et = [etas[i] if lmr[i] else None for i in range(n)]
    p_enc = rd.Plan([rd.make_job(P[i], *imgs[i].shape, src=d_img[i], dst=marked[i], map_bits=lm[i], eta_bits=et[i],
                                 payload=d_pay[i], nbits=caps[i], info=info[i]) for i in range(n)], st)
    p_dec = rd.Plan([rd.make_job(P[i], *imgs[i].shape, src=marked[i], dst=rec[i], map_bits=lm[i], eta_bits=et[i],
                                 bits_out=bits[i], max_bits=caps[i], info=info[i], b=0) for i in range(n)], st)
    torch.cuda.synchronize()
    for _ in range(3):
        p_enc.run(rd.OP_ENCODE, st)
        p_dec.run(rd.OP_DECODE, st)
    torch.cuda.synchronize()
    assert p_enc.status(st) == 0 and p_dec.status(st) == 0
    for i in range(n):
        op = oracle.Params(variant=variants[i], **_keys(seeds[i]))
        r = oracle.label_encrypt(op, imgs[i])
        l_np = r.map_bits if lmr[i] else None
        mref, _ = oracle.embed(op, r.b, r.enc, pays[i], r.capacity, l_np)
        assert np.array_equal(marked[i].cpu().numpy(), mref), i
        xref, xk = oracle.extract(op, r.b, mref, r.capacity, l_np)
        assert np.array_equal(_bits(bits[i], xk), xref), i
        rref = oracle.decrypt_recover(op, r.b, mref, l_np, r.eta_bits if lmr[i] else None)
        assert np.array_equal(rec[i].cpu().numpy(), rref), i


def test_full_benchmark_batch_sampled(rd):
    """The benchmark's own workload and launch configuration -- 1000 synthetic 512 x 512
    images, EMR (even) / LMR (odd) with ceil(N/8) side bits, full-capacity payloads,
    one plan per operation over the whole batch, jobs built as bench.py builds them --
    and a sample of its images checked against the oracle output by output."""
    import bench
    n, H, W = 1000, 512, 512
    N = H * W
    imgs_np = bench.make_images(n, H, W)              # the benchmark's generator (a spawned pool)
    variants = [rd.EMR if k % 2 == 0 else rd.LMR for k in range(n)]
    lmr = [(v & 1) == rd.LMR for v in variants]
    params = [rd.Params(variant=variants[k], **{f: bench.image_keys(k)[f] for f in ("k1", "nonce1", "k2", "nonce2")})
              for k in range(n)]
    imgs = torch.from_numpy(imgs_np).cuda()
    enc, marked, rec = torch.empty_like(imgs), torch.empty_like(imgs), torch.empty_like(imgs)
    mb = ((N + 31) // 32) * 4
    maps = torch.zeros((n, mb), dtype=torch.uint8, device="cuda")
    etas = torch.zeros((n, mb), dtype=torch.uint8, device="cuda")
    sn = bench.side_nbits(H, W)
    side_np = np.zeros((n, ((sn + 31) // 32) * 4), np.uint8)
    for k in range(n):
        if lmr[k]:
            b = synth.random_bits(k, sn)
            side_np[k, :b.size] = b
    sides = torch.from_numpy(side_np).cuda()
    info = rd.new_info(n)
    rd.Plan([rd.make_job(params[k], H, W, src=imgs[k], dst=enc[k], map_bits=maps[k] if lmr[k] else None,
                         eta_bits=etas[k] if lmr[k] else None, side_bits=sides[k] if lmr[k] else None,
                         side_nbits=sn if lmr[k] else 0, info=info[k]) for k in range(n)]).run(rd.OP_LABEL_ENCRYPT)
    torch.cuda.synchronize()
    caps = [r["capacity"] for r in rd.read_info(info)]
    pb = ((7 * N + 31) // 32) * 4
    pay_np = np.zeros((n, pb), np.uint8)
    for k in range(n):
        b = synth.payload_bits(synth.image_seed(bench.BASE_SEED, k), caps[k])
        pay_np[k, :b.size] = b
    payload = torch.from_numpy(pay_np).cuda()
    bits = torch.zeros((n, pb), dtype=torch.uint8, device="cuda")
    m = [maps[k] if lmr[k] else None for k in range(n)]
    rd.Plan([rd.make_job(params[k], H, W, src=enc[k], dst=marked[k], map_bits=m[k], payload=payload[k],
                         nbits=caps[k], info=info[k], b=0) for k in range(n)]).run(rd.OP_EMBED)
    rd.Plan([rd.make_job(params[k], H, W, src=marked[k], map_bits=m[k], bits_out=bits[k], max_bits=caps[k],
                         info=info[k], b=0) for k in range(n)]).run(rd.OP_EXTRACT)
    rd.Plan([rd.make_job(params[k], H, W, src=marked[k], dst=rec[k], map_bits=m[k],
                         eta_bits=etas[k] if lmr[k] else None, info=info[k], b=0)
             for k in range(n)]).run(rd.OP_DECRYPT_RECOVER)
    torch.cuda.synchronize()
    got = rd.read_info(info)
    sample = sorted({0, 1, 2, 3, 498, 499, 998, 999} | set(np.random.default_rng(7).integers(0, n, 8).tolist()))
    for k in sample:
        v = variants[k]
        op = oracle.Params(variant=v, **{f: bench.image_keys(k)[f] for f in ("k1", "nonce1", "k2", "nonce2")})
        side = synth.random_bits(k, sn) if lmr[k] else None
        r = oracle.label_encrypt(op, imgs_np[k], side, sn if lmr[k] else 0)
        g = got[k]
        assert g["hist"] == [int(x) for x in r.hist] and g["b"] == r.b and g["capacity"] == r.capacity, k
        assert np.array_equal(enc[k].cpu().numpy(), r.enc), k
        lm = r.map_bits if lmr[k] else None
        if lmr[k]:
            assert np.array_equal(_bits(maps[k], N), r.map_bits), k
            assert np.array_equal(_bits(etas[k], N), r.eta_bits), k
        mref, emb = oracle.embed(op, r.b, r.enc, pay_np[k, :(r.capacity + 7) // 8], r.capacity, lm)
        assert g["embedded"] == emb and np.array_equal(marked[k].cpu().numpy(), mref), k
        xref, xk = oracle.extract(op, r.b, mref, r.capacity, lm)
        assert g["extracted"] == xk and np.array_equal(_bits(bits[k], xk), xref), k
        rref = oracle.decrypt_recover(op, r.b, mref, lm, r.eta_bits if lmr[k] else None)
        assert np.array_equal(rec[k].cpu().numpy(), rref), k

    # the fused calls in the benchmark's launch configuration (one plan per call over the
    # whole batch, jobs as bench.py builds them): every image equals the separable chain's
    # output checked above
    marked2, rec2 = torch.empty_like(imgs), torch.empty_like(imgs)
    maps2 = torch.zeros_like(maps)
    etas2 = torch.zeros_like(etas)
    bits2 = torch.zeros_like(bits)
    info2 = rd.new_info(n)
    m2 = [maps2[k] if lmr[k] else None for k in range(n)]
    pe = rd.Plan([rd.make_job(params[k], H, W, src=imgs[k], dst=marked2[k], map_bits=m2[k],
                              eta_bits=etas2[k] if lmr[k] else None, side_bits=sides[k] if lmr[k] else None,
                              side_nbits=sn if lmr[k] else 0, payload=payload[k], nbits=caps[k], info=info2[k])
                  for k in range(n)])
    pd = rd.Plan([rd.make_job(params[k], H, W, src=marked2[k], dst=rec2[k], map_bits=m2[k],
                              eta_bits=etas2[k] if lmr[k] else None, bits_out=bits2[k], max_bits=caps[k],
                              info=info2[k], b=0) for k in range(n)])
    for _ in range(2):
        pe.run(rd.OP_ENCODE)
        pd.run(rd.OP_DECODE)
    torch.cuda.synchronize()
    assert pe.status() == 0 and pd.status() == 0
    assert torch.equal(marked2, marked) and torch.equal(rec2, rec) and torch.equal(bits2, bits)
    assert torch.equal(maps2, maps) and torch.equal(etas2, etas)
    g2 = rd.read_info(info2)
    assert all(g2[k]["embedded"] == caps[k] and g2[k]["extracted"] == caps[k] and g2[k]["b"] == got[k]["b"]
               for k in range(n))
