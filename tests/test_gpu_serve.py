"""Serving loop: requests admitted while others are on the GPU (continuous batching over
several streams) give the same bytes as the same requests served one at a time, and
those bytes match the CPU oracle."""
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


def _pin(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def _encode_requests(rd, sv, n, seed0):
    rng = np.random.default_rng(seed0)
    reqs = []
    for i in range(n):
        H, W = int(rng.integers(40, 700)), int(rng.integers(40, 700))
        seed = seed0 * 1000 + i
        k = synth.keys(seed)
        p = rd.Params(variant=rd.EMR if i % 2 == 0 else rd.LMR, k1=k["k1"], nonce1=k["nonce1"], k2=k["k2"],
                      nonce2=k["nonce2"])
        img = synth.synth_image(H, W, seed, noise_sigma=2.0)
        nbits = H * W // 3
        reqs.append(sv.Request(rid=i, kind="encode", params=p, image=_pin(img),
                               payload=_pin(synth.payload_bits(seed, nbits)), nbits=nbits))
    return reqs


def _clone(sv, r):
    return sv.Request(rid=r.rid, kind=r.kind, params=r.params, image=r.image, payload=r.payload, nbits=r.nbits, b=r.b,
                      lmr_map=r.lmr_map, lmr_eta=r.lmr_eta, arrival=r.arrival, state=r.state,
                      keep_state=r.keep_state)


def _same(a, b):
    keys = set(a.result) - {"info"}
    assert keys == set(b.result) - {"info"}
    for k in keys:
        assert torch.equal(a.result[k], b.result[k]), (a.rid, k)
    for f in ("b", "capacity", "embedded", "extracted", "hist"):
        assert a.result["info"][f] == b.result["info"][f], (a.rid, f)


def test_mixed_equals_alone(mods):
    rd, sv = mods
    enc = _encode_requests(rd, sv, 14, 7)
    # decode requests from one-at-a-time encodes
    alone_enc = [sv.Server(max_batch=1, streams=1).run([_clone(sv, r)], realtime=False)[0] for r in enc]
    dec = []
    for r, a in zip(enc, alone_enc):
        inf = a.result["info"]
        dec.append(sv.Request(rid=100 + r.rid, kind="decode", params=r.params, image=a.result["marked"],
                              nbits=inf["embedded"], b=inf["b"], lmr_map=a.result.get("map_bits"),
                              lmr_eta=a.result.get("eta_bits")))
    mixed = [_clone(sv, r) for r in enc + dec]
    rng = np.random.default_rng(1)
    for r in mixed:
        r.arrival = float(rng.uniform(0, 0.02))          # arrive while earlier work runs
    srv = sv.Server(max_batch=5, streams=3)
    out = {r.rid: r for r in srv.run(mixed, realtime=True)}
    assert len(out) == len(mixed)
    for r in enc + dec:
        alone = sv.Server(max_batch=1, streams=1).run([_clone(sv, r)], realtime=False)[0]
        _same(out[r.rid], alone)
    # LMR decode is lossless, EMR loses the LSB plane only, messages come back
    for r in dec:
        got = out[r.rid].result
        src = enc[r.rid - 100]
        img = src.image.numpy()
        rec = got["recovered"].numpy()
        if r.params.variant == rd.LMR:
            assert np.array_equal(rec, img)
        else:
            assert not ((rec ^ img) & 0xFE).any()
        nb = r.nbits // 8
        assert torch.equal(got["bits"][:nb], src.payload[:nb])
    st = sv.latency_stats(list(out.values()))
    assert st["requests"] == len(mixed) and st["p99_ms"] >= st["p50_ms"] > 0


def test_served_encode_matches_oracle(mods):
    rd, sv = mods
    r = _encode_requests(rd, sv, 2, 11)[1]                 # an LMR request
    got = sv.Server().run([r], realtime=False)[0].result
    op = oracle.Params(variant=r.params.variant, k1=r.params.k1, nonce1=r.params.nonce1, k2=r.params.k2,
                       nonce2=r.params.nonce2)
    img = r.image.numpy()
    e = oracle.label_encrypt(op, img)
    marked, k = oracle.embed(op, e.b, e.enc, r.payload.numpy(), r.nbits, e.map_bits)
    assert got["info"]["b"] == e.b and got["info"]["embedded"] == k
    assert np.array_equal(got["marked"].numpy(), marked)


def test_budget_admission(mods):
    rd, sv = mods
    reqs = _encode_requests(rd, sv, 6, 3)
    one = max(r.device_bytes() for r in reqs)
    srv = sv.Server(budget_bytes=one * 1.5, max_batch=8, streams=4)   # at most one request in flight
    done = srv.run(reqs, realtime=False)
    assert len(done) == 6 and srv.in_use == pytest.approx(0.0)


def test_device_resident_maps_and_admission_window(mods):
    """Encodes that keep their LMR maps on the device hand back a handle instead of host
    maps; decodes that name the handle read the maps in place and give the same bytes
    as decodes fed the maps from the host, with the server's admission window on."""
    rd, sv = mods
    enc = _encode_requests(rd, sv, 10, 21)
    srv = sv.Server(max_batch=8, streams=2, admit_window_ms=2.0)
    kept = []
    for r in enc:
        c = _clone(sv, r)
        c.keep_state = True
        c.arrival = 0.0                             # all at once: they cannot all go one by one
        kept.append(c)
    done = {r.rid: r for r in srv.run(kept, realtime=True)}
    assert max(b["requests"] for b in srv.batches) > 1, "no two requests left together"
    ref = {r.rid: sv.Server(max_batch=1, streams=1).run([_clone(sv, r)], realtime=False)[0] for r in enc}
    dec_state, dec_host = [], []
    for r in enc:
        got, alone = done[r.rid].result, ref[r.rid].result
        assert torch.equal(got["marked"], alone["marked"])
        inf = got["info"]
        lmr = r.params.variant == rd.LMR
        if lmr:
            assert got.get("state") and "map_bits" not in got
            assert srv.state.get(got["state"]) is not None
        else:
            assert not got.get("state")
        dec_state.append(sv.Request(rid=100 + r.rid, kind="decode", params=r.params, image=got["marked"],
                                    nbits=inf["embedded"], b=inf["b"], state=got.get("state", 0)))
        dec_host.append(sv.Request(rid=200 + r.rid, kind="decode", params=r.params, image=alone["marked"],
                                   nbits=inf["embedded"], b=inf["b"], lmr_map=alone.get("map_bits"),
                                   lmr_eta=alone.get("eta_bits")))
    in_state = srv.state.bytes
    assert in_state > 0
    out = {r.rid: r for r in srv.run(dec_state, realtime=False)}
    for a, b in zip(dec_state, dec_host):
        ra = out[a.rid].result
        rb = sv.Server().run([b], realtime=False)[0].result
        assert torch.equal(ra["bits"], rb["bits"]) and torch.equal(ra["recovered"], rb["recovered"]), a.rid
        if a.params.variant == rd.LMR:
            assert np.array_equal(ra["recovered"].numpy(), enc[a.rid - 100].image.numpy())
    # the store is charged to the admission budget and can be emptied
    for r in enc:
        h = done[r.rid].result.get("state")
        if h:
            srv.drop_state(h)
    assert srv.state.bytes == 0 and srv.ex.state_bytes() == 0
