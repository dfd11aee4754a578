"""GPU parity of the related-work MED variants (RDHEI_EMR_MED / RDHEI_LMR_MED): the
owner's MED labels and histogram, and the receiver's tiled anti-diagonal wavefront
recovery, byte for byte against the oracle; mixed with the paper's variants in one
batch; the wavefront's done flags leave no error behind."""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_07992_gb300 import synth
from test_gpu_parity import _pipeline

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rd():
    from paper_2302_07992_gb300 import rdhei
    return rdhei


SHAPES = [(64, 64), (96, 160), (100, 130), (1, 50), (50, 1), (3, 3), (33, 129), (31, 127), (257, 333),
          (512, 512), (128, 1024), (2, 2)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("variant", [oracle.EMR_MED, oracle.LMR_MED])
def test_med_pipeline_shapes(rd, shape, variant):
    H, W = shape
    seed = H * 1000 + W + 7 * variant
    img = synth.synth_image(H, W, seed)
    _pipeline(rd, img, variant, seed)


@pytest.mark.parametrize("variant", [oracle.EMR_MED, oracle.LMR_MED])
@pytest.mark.parametrize("kw", [dict(rot_enable=0), dict(rot_lmin=2), dict(b=3), dict(b=6)])
def test_med_pipeline_parameters(rd, variant, kw):
    img = synth.synth_image(200, 264, 11, noise_sigma=2.0)
    _pipeline(rd, img, variant, 19, **kw)


def test_med_edge_images(rd):
    const = np.full((70, 140), 91, np.uint8)
    i, j = np.mgrid[0:90, 0:200]
    plane = (100 + i - j).astype(np.uint8)
    stripes = np.tile(np.array([0, 255], np.uint8), (70, 90))
    noise = np.random.default_rng(3).integers(0, 256, size=(160, 160)).astype(np.uint8)
    for k, img in enumerate((const, plane, stripes, noise)):
        for variant in (oracle.EMR_MED, oracle.LMR_MED):
            _pipeline(rd, img, variant, 40 + k)


def test_med_large_image_many_diagonals(rd):
    """2048 x 1536: 64 x 12 wavefront tiles, 75 anti-diagonals."""
    img = synth.synth_image(2048, 1536, 77)
    _pipeline(rd, img, oracle.LMR_MED, 77)


def test_mixed_batch_in_one_plan(rd):
    """Paper variants and MED variants of uneven sizes in one batch, through the
    batched pipeline: each image's outputs equal its own oracle run."""
    from paper_2302_07992_gb300 import pipeline as pp
    shapes = [(96, 160), (257, 333), (64, 64), (130, 70), (512, 512), (33, 129), (200, 72), (1, 90)]
    variants = [rd.EMR, rd.LMR, rd.EMR_MED, rd.LMR_MED] * 2
    imgs, params, oparams, seeds = [], [], [], []
    for k, ((H, W), v) in enumerate(zip(shapes, variants)):
        seed = 900 + k
        kk = synth.keys(seed)
        common = dict(variant=v, k1=kk["k1"], nonce1=kk["nonce1"], k2=kk["k2"], nonce2=kk["nonce2"])
        imgs.append(synth.synth_image(H, W, seed))
        params.append(rd.Params(**common))
        oparams.append(oracle.Params(**common))
        seeds.append(seed)
    s = pp.ImageSet(imgs, variants, params)
    bp = pp.BatchedPipeline(s, pp.default_payload(lambda i: seeds[i]))
    bp.step()
    torch.cuda.synchronize()
    for i in range(len(imgs)):
        lmr = (variants[i] & 1) == rd.LMR
        r = oracle.label_encrypt(oparams[i], imgs[i])
        assert np.array_equal(s.enc[i].cpu().numpy(), r.enc), i
        pay = s.payload[i].cpu().numpy()
        lm = r.map_bits if lmr else None
        mref, _ = oracle.embed(oparams[i], r.b, r.enc, pay, r.capacity, lm)
        assert np.array_equal(s.marked[i].cpu().numpy(), mref), i
        rref = oracle.decrypt_recover(oparams[i], r.b, mref, lm, r.eta_bits if lmr else None)
        assert np.array_equal(s.rec[i].cpu().numpy(), rref), i
    # the wavefront stage ran and its waits all succeeded
    dec_plan = [pl for pl, op in bp.plans if op == rd.OP_DECRYPT_RECOVER][0]
    assert 3 in dec_plan.active_stages(rd.OP_DECRYPT_RECOVER)
    assert dec_plan.status() == 0


@pytest.mark.parametrize("cols", [0, 64, 128, 256])
@pytest.mark.parametrize("shape", [(200, 530), (1100, 70), (37, 1000), (600, 333)])
def test_wave_widths_agree(rd, cols, shape):
    """The row-band pipeline (0) and every tile width recover the oracle's image; the
    wavefront stage can be rerun on restaged pixels (it clears its own flags and
    ticket).  1100 rows = 35 bands: three rounds of the 16-warp band pipeline."""
    H, W = shape
    img = synth.synth_image(H, W, 61)
    for variant in (oracle.EMR_MED, oracle.LMR_MED):
        k = synth.keys(61)
        common = dict(variant=variant, k1=k["k1"], nonce1=k["nonce1"], k2=k["k2"], nonce2=k["nonce2"])
        p, op = rd.Params(**common), oracle.Params(**common)
        lmr = (variant & 1) == rd.LMR
        e = oracle.label_encrypt(op, img)
        pay = synth.payload_bits(61, e.capacity)
        lm = e.map_bits if lmr else None
        marked, _ = oracle.embed(op, e.b, e.enc, pay, e.capacity, lm)
        ref = oracle.decrypt_recover(op, e.b, marked, lm, e.eta_bits if lmr else None)
        dev_marked = torch.from_numpy(marked).cuda()
        out = torch.empty_like(dev_marked)
        mb = rd.as_bitbuf(torch.from_numpy(e.map_bits), H * W) if lmr else None
        eb = rd.as_bitbuf(torch.from_numpy(e.eta_bits), H * W) if lmr else None
        info = rd.new_info(1)
        job = rd.make_job(p, H, W, src=dev_marked, dst=out, map_bits=mb, eta_bits=eb, info=info, b=e.b)
        plan = rd.Plan([job], wave_cols=cols)
        plan.run(rd.OP_DECRYPT_RECOVER)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref)
        for _ in range(2):
            plan.run_stage(rd.OP_DECRYPT_RECOVER, 2)
            plan.run_stage(rd.OP_DECRYPT_RECOVER, 3)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref)
        assert plan.status() == 0


def test_autotuner_picks_and_caches_a_width(rd):
    from paper_2302_07992_gb300 import tune
    H, W = 256, 512
    jobs, keep = [], []
    for i in range(4):
        img = synth.synth_image(H, W, 80 + i)
        k = synth.keys(80 + i)
        p = rd.Params(variant=rd.EMR_MED, k1=k["k1"], nonce1=k["nonce1"], k2=k["k2"], nonce2=k["nonce2"])
        e = rd.label_encrypt(torch.from_numpy(img).cuda(), p)
        out = torch.empty_like(e["enc"])
        info = rd.new_info(1)
        keep += [e, out, info]
        jobs.append(rd.make_job(p, H, W, src=e["enc"], dst=out, info=info, b=e["b"]))
    best, times = tune.best_wave_cols(jobs, refresh=True)
    assert best in tune.WAVE_WIDTHS and set(times) == {str(c) for c in tune.WAVE_WIDTHS}
    assert all(v > 0 for v in times.values())
    again, cached = tune.best_wave_cols(jobs)
    assert again == best and cached == times
