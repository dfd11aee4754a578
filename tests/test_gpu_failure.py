"""Failure detection on the GPU without a fault: a bounded device-side wait on a flag
that nothing sets gives up after its limit and reports RDHEI_ETIMEOUT, the context
stays usable, and the serving loop turns a request the library rejects into an
"error" status while it serves the others."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2302_07992_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2302_07992_gb300 import rdhei, serve
    return rdhei, serve


def test_bounded_wait_times_out_and_context_survives(mods):
    rd, _ = mods
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")          # nothing sets it
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    assert rd.wait_selftest(flag, 50_000_000) == rd.RDHEI_ETIMEOUT
    dt = time.perf_counter() - t0
    assert 0.045 <= dt < 1.5, dt
    flag.fill_(1)
    assert rd.wait_selftest(flag, 50_000_000) == rd.RDHEI_OK
    # the context still runs the path, byte-exact against the oracle
    H, W, seed = 70, 90, 11
    img = synth.synth_image(H, W, seed)
    k = synth.keys(seed)
    p = rd.Params(variant=rd.LMR, k1=k["k1"], nonce1=k["nonce1"], k2=k["k2"], nonce2=k["nonce2"])
    op = oracle.Params(variant=oracle.LMR, k1=k["k1"], nonce1=k["nonce1"], k2=k["k2"], nonce2=k["nonce2"])
    e = rd.label_encrypt(torch.from_numpy(img).cuda(), p)
    assert np.array_equal(e["enc"].cpu().numpy(), oracle.label_encrypt(op, img).enc)


def test_selftest_rejects_bad_pointers(mods):
    rd, _ = mods
    import ctypes
    st = torch.cuda.current_stream().cuda_stream
    s = torch.zeros(2, dtype=torch.int32, device="cuda")
    assert rd._lib.rdhei_wait_selftest(None, 10, ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(st)) == rd.RDHEI_EINVAL
    assert rd._lib.rdhei_wait_selftest(ctypes.c_void_p(s.data_ptr() + 2), 10, ctypes.c_void_p(s.data_ptr()),
                                       ctypes.c_void_p(st)) == rd.RDHEI_EINVAL


def test_serving_marks_a_rejected_batch_and_serves_the_rest(mods):
    rd, sv = mods
    reqs = []
    for i in range(6):
        seed = 500 + i
        k = synth.keys(seed)
        img = synth.synth_image(64, 80, seed)
        nbits = 1000
        # request 3 asks for an unknown variant: the library rejects its plan (EINVAL)
        p = rd.Params(variant=7 if i == 3 else rd.EMR, k1=k["k1"], nonce1=k["nonce1"], k2=k["k2"], nonce2=k["nonce2"])
        reqs.append(sv.Request(rid=i, kind="encode", params=p, image=torch.from_numpy(img).pin_memory(),
                               payload=torch.from_numpy(synth.payload_bits(seed, nbits)).pin_memory(), nbits=nbits))
    srv = sv.Server(max_batch=2, streams=2)
    srv.run(reqs, realtime=False)
    st = {r.rid: r.status for r in reqs}
    assert st[2] == st[3] == "error" and "EINVAL" in reqs[3].error
    assert all(st[i] == "ok" for i in (0, 1, 4, 5))
    assert srv.in_use == pytest.approx(0.0) and len(srv.ex.free_streams) == 2
    m = srv.metrics()
    assert m["status"]["error"] == 2 and m["status"]["ok"] == 4
