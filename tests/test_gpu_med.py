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
