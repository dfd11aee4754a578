"""The autotuner's knobs change launch shapes only: every value of every tuned plan
parameter gives outputs equal to the oracle's, byte for byte, and the tuner picks one
of its candidates and caches it."""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_07992_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2302_07992_gb300 import rdhei, tune
    return rdhei, tune


def _keys(seed):
    k = synth.keys(seed)
    return dict(k1=k["k1"], nonce1=k["nonce1"], k2=k["k2"], nonce2=k["nonce2"])


# wide images (many chunks per strip), ragged strips, a strip shorter than every part
SHAPES = [(200, 4100), (130, 2050), (64, 1000), (257, 333), (5, 700), (512, 512)]
VARIANTS = [0, 1, 2, 1, 0, 3]


@pytest.fixture(scope="module")
def batch(mods):
    rd, _ = mods
    n = len(SHAPES)
    imgs = [synth.synth_image(H, W, 1300 + i) for i, (H, W) in enumerate(SHAPES)]
    P = [rd.Params(variant=VARIANTS[i], **_keys(1300 + i)) for i in range(n)]
    refs = []
    for i in range(n):
        op = oracle.Params(variant=VARIANTS[i], **_keys(1300 + i))
        lmr = (VARIANTS[i] & 1) == 1
        r = oracle.label_encrypt(op, imgs[i])
        pay = synth.payload_bits(1300 + i, r.capacity)
        lm = r.map_bits if lmr else None
        marked, _ = oracle.embed(op, r.b, r.enc, pay, r.capacity, lm)
        xref, xk = oracle.extract(op, r.b, marked, r.capacity, lm)
        rref = oracle.decrypt_recover(op, r.b, marked, lm, r.eta_bits if lmr else None)
        refs.append(dict(r=r, pay=pay, marked=marked, bits=xref, nbits=xk, rec=rref, lmr=lmr))
    return imgs, P, refs


@pytest.mark.parametrize("rows", [64, 32, 16, 8, 4])
def test_every_extraction_split_matches_the_oracle(mods, batch, rows):
    rd, _ = mods
    imgs, P, refs = batch
    n = len(imgs)
    marked = [torch.from_numpy(ref["marked"]).cuda() for ref in refs]
    rec = [torch.empty_like(m) for m in marked]
    bits = [rd.bitbuf(ref["r"].capacity) for ref in refs]
    for b in bits:
        b.fill_(0xA5)                                   # stale bytes must not leak into the result
    maps = [rd.as_bitbuf(torch.from_numpy(ref["r"].map_bits), imgs[i].size) if ref["lmr"] else None
            for i, ref in enumerate(refs)]
    etas = [rd.as_bitbuf(torch.from_numpy(ref["r"].eta_bits), imgs[i].size) if ref["lmr"] else None
            for i, ref in enumerate(refs)]
    info = rd.new_info(n)
    jobs = []
    for i, ref in enumerate(refs):
        H, W = imgs[i].shape
        jobs.append(rd.make_job(P[i], H, W, src=marked[i], dst=rec[i], map_bits=maps[i], eta_bits=etas[i],
                                bits_out=bits[i], max_bits=ref["r"].capacity, info=info[i], b=ref["r"].b))
    plan = rd.Plan(jobs, params={rd.PARAM_EXTRACT_ROWS: rows})
    assert plan.get_param(rd.PARAM_EXTRACT_ROWS) == rows
    for _ in range(2):
        plan.run(rd.OP_DECODE)
    torch.cuda.synchronize()
    assert plan.status() == 0
    for i, ref in enumerate(refs):
        got = bits[i].cpu().numpy()
        assert np.array_equal(got[: (ref["nbits"] + 7) // 8], ref["bits"]), (rows, i)
        assert not got[(ref["nbits"] + 7) // 8:].any(), (rows, i)
        assert np.array_equal(rec[i].cpu().numpy(), ref["rec"]), (rows, i)


@pytest.mark.parametrize("split", [1, 3, 8, 64])
def test_every_encode_split_matches_the_oracle(mods, batch, split):
    rd, _ = mods
    imgs, P, refs = batch
    n = len(imgs)
    d_img = [torch.from_numpy(im).cuda() for im in imgs]
    enc = [torch.empty_like(x) for x in d_img]
    maps = [rd.bitbuf(im.size) for im in imgs]
    info = rd.new_info(n)
    jobs = [rd.make_job(P[i], *imgs[i].shape, src=d_img[i], dst=enc[i], map_bits=maps[i], info=info[i])
            for i in range(n)]
    plan = rd.Plan(jobs, params={rd.PARAM_ENC_SPLIT: split})
    plan.run(rd.OP_LABEL_ENCRYPT)
    torch.cuda.synchronize()
    for i, ref in enumerate(refs):
        assert np.array_equal(enc[i].cpu().numpy(), ref["r"].enc), (split, i)
        assert np.array_equal(maps[i].cpu().numpy()[: (imgs[i].size + 7) // 8], ref["r"].map_bits), (split, i)


def test_tuner_picks_and_caches_a_candidate(mods, batch, tmp_path, monkeypatch):
    rd, tune = mods
    monkeypatch.setattr(tune, "_CACHE", str(tmp_path / "cache.json"))
    imgs, P, refs = batch
    n = len(imgs)
    d_img = [torch.from_numpy(im).cuda() for im in imgs]
    enc = [torch.empty_like(x) for x in d_img]
    info = rd.new_info(n)
    enc_jobs = [rd.make_job(P[i], *imgs[i].shape, src=d_img[i], dst=enc[i], info=info[i]) for i in range(n)]
    best, times = tune.best_enc_split(enc_jobs)
    assert best in tune.ENC_SPLITS and set(times) == {str(v) for v in tune.ENC_SPLITS}
    again, cached = tune.best_enc_split(enc_jobs)
    assert again == best and cached == times                # from the cache
    marked = [torch.from_numpy(ref["marked"]).cuda() for ref in refs]
    rec = [torch.empty_like(m) for m in marked]
    bits = [rd.bitbuf(ref["r"].capacity) for ref in refs]
    maps = [rd.as_bitbuf(torch.from_numpy(ref["r"].map_bits), imgs[i].size) if ref["lmr"] else None
            for i, ref in enumerate(refs)]
    etas = [rd.as_bitbuf(torch.from_numpy(ref["r"].eta_bits), imgs[i].size) if ref["lmr"] else None
            for i, ref in enumerate(refs)]
    dec_jobs = [rd.make_job(P[i], *imgs[i].shape, src=marked[i], dst=rec[i], map_bits=maps[i], eta_bits=etas[i],
                            bits_out=bits[i], max_bits=refs[i]["r"].capacity, info=info[i], b=refs[i]["r"].b)
                for i in range(n)]
    rows, t2 = tune.best_extract_rows(dec_jobs)
    assert rows in tune.EXTRACT_ROWS and set(t2) == {str(v) for v in tune.EXTRACT_ROWS}
    # and the tuned configuration still gives the oracle's bytes
    plan = rd.Plan(dec_jobs, params={rd.PARAM_EXTRACT_ROWS: rows})
    plan.run(rd.OP_DECODE)
    torch.cuda.synchronize()
    for i, ref in enumerate(refs):
        assert np.array_equal(bits[i].cpu().numpy()[: (ref["nbits"] + 7) // 8], ref["bits"]), i
        assert np.array_equal(rec[i].cpu().numpy(), ref["rec"]), i


def test_bad_parameter_values_are_rejected(mods):
    rd, _ = mods
    p = rd.Params()
    img = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    plan = rd.Plan([rd.make_job(p, 64, 64, src=img, dst=torch.empty_like(img), info=rd.new_info(1))])
    for param, value in ((rd.PARAM_EXTRACT_ROWS, 12), (rd.PARAM_EXTRACT_ROWS, 128), (rd.PARAM_ENC_SPLIT, 65),
                         (rd.PARAM_ENC_SPLIT, -1), (99, 1), (rd.PARAM_WAVE_COLS, 64)):
        with pytest.raises(rd.RdheiError):
            plan.set_param(param, value)                # wave width: only before upload
