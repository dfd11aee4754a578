"""The serving scheduler on the CPU: a host-thread executor stands in for the GPU, with
injected delays and failures.  Nothing here launches a kernel; the scheduler's
admission, batching, cancellation, failure and metrics logic is the code under test."""
import json
import threading
import time

import numpy as np
import pytest

from paper_2302_07992_gb300.sched import LAT_EDGES_MS, STATUSES, Request, Scheduler, latency_stats


class FakeBatch:
    def __init__(self, reqs, delay, fail):
        self.reqs = reqs
        self.fail = fail
        self.done = threading.Event()
        self.timer = threading.Timer(delay, self.done.set)
        self.timer.start()


class FakeExecutor:
    """Completes each batch on a timer thread after delay(reqs) seconds.  Injected
    faults: launch_fail(reqs) -> raise at launch; batch_fail(reqs) -> results() raises
    (a device-side error reported at completion).  Records what it ran and what it
    gave back."""

    def __init__(self, slots=2, delay=lambda reqs: 0.002, launch_fail=None, batch_fail=None, capacity=None):
        self.slots = slots
        self.delay = delay
        self.launch_fail = launch_fail or (lambda reqs: False)
        self.batch_fail = batch_fail or (lambda reqs: False)
        self.capacity = capacity or (lambda r: 10 ** 9)
        self.launched, self.discarded, self.released = [], [], 0
        self.live = 0
        self.max_live = 0

    def launch(self, reqs):
        if self.launch_fail(reqs):
            raise RuntimeError("injected launch failure")
        self.launched.append([r.rid for r in reqs])
        self.live += 1
        self.max_live = max(self.max_live, self.live)
        assert self.live <= self.slots
        return FakeBatch(reqs, self.delay(reqs), self.batch_fail(reqs))

    def ready(self, h):
        return h.done.is_set()

    def wait(self, h):
        assert h.done.wait(10.0)

    def results(self, h):
        if h.fail:
            raise RuntimeError("injected device error ETIMEOUT")
        out = []
        for r in h.reqs:
            cap = self.capacity(r)
            emb = min(r.nbits, cap)
            out.append({"buf": f"result-{r.rid}",
                        "info": {"b": 1 + r.rid % 8, "capacity": cap, "embedded": emb, "extracted": 0,
                                 "hist": [0] * 9, "status": 2 if r.nbits > cap else 0}})
        return out

    def discard(self, result):
        self.discarded.append(result["buf"])

    def release(self, h):
        self.live -= 1
        self.released += 1


def _reqs(n, kinds=("encode",), side=64, nbits=100, spacing=0.0, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        H = W = side if side else int(rng.integers(16, 256))
        out.append(Request(rid=i, kind=kinds[i % len(kinds)], params=None, image=np.zeros((H, W), np.uint8),
                           nbits=nbits, arrival=i * spacing))
    return out


def _check_terminal(sched, reqs, ex):
    """Every request ends in exactly one status; budget and slots are all given back."""
    assert sorted(r.rid for r in sched.completed) == sorted(r.rid for r in reqs)
    assert all(r.status in STATUSES and r.done >= 0 for r in reqs)
    assert sched.in_use == pytest.approx(0.0)
    assert not sched.inflight and not sched.queue
    assert ex.live == 0 and ex.released == len(ex.launched)


def test_all_served_in_batches_of_one_kind():
    ex = FakeExecutor(slots=3)
    reqs = _reqs(40, kinds=("encode", "encode", "decode"))
    s = Scheduler(ex, max_batch=8)
    done = s.run(reqs, realtime=False)
    _check_terminal(s, reqs, ex)
    assert all(r.status == "ok" for r in done)
    kind = {r.rid: r.kind for r in reqs}
    for b in ex.launched:
        assert len(b) <= 8 and len({kind[i] for i in b}) == 1
    assert sorted(i for b in ex.launched for i in b) == list(range(40))
    assert ex.max_live <= 3


def test_batches_keep_arrival_order_within_a_kind():
    ex = FakeExecutor(slots=1)
    reqs = _reqs(30, kinds=("encode",))
    s = Scheduler(ex, max_batch=7)
    s.run(reqs, realtime=False)
    flat = [i for b in ex.launched for i in b]
    assert flat == sorted(flat)


def test_budget_limits_requests_in_flight():
    """With a budget of 1.5 requests only one request is ever in flight, although the
    executor has four slots; a request larger than the whole budget still runs alone."""
    reqs = _reqs(6)
    one = reqs[0].device_bytes()
    live = []

    class Watch(FakeExecutor):
        def launch(self, rs):
            live.append(sum(len(b.reqs) for b in self.batches_live) + len(rs))
            h = super().launch(rs)
            self.batches_live.append(h)
            return h

        def release(self, h):
            self.batches_live.remove(h)
            super().release(h)

    ex = Watch(slots=4)
    ex.batches_live = []
    s = Scheduler(ex, budget_bytes=1.5 * one, max_batch=8)
    s.run(reqs, realtime=False)
    _check_terminal(s, reqs, ex)
    assert max(live) == 1
    big = _reqs(2, side=512)
    ex2 = FakeExecutor(slots=2)
    s2 = Scheduler(ex2, budget_bytes=0.5 * big[0].device_bytes())
    s2.run(big, realtime=False)
    _check_terminal(s2, big, ex2)
    assert all(r.status == "ok" for r in big) and ex2.max_live == 1


def test_pixel_cap_splits_batches():
    ex = FakeExecutor(slots=1)
    reqs = _reqs(10, side=100)
    s = Scheduler(ex, max_batch=64, max_batch_pixels=3 * 100 * 100)
    s.run(reqs, realtime=False)
    assert [len(b) for b in ex.launched] == [3, 3, 3, 1]


def test_cancel_queued_and_in_flight():
    """A cancelled queued request never runs; an in-flight one runs and its result is
    discarded (its buffers handed back), and neither reaches consume()."""
    ex = FakeExecutor(slots=1, delay=lambda reqs: 0.05)
    reqs = _reqs(6)
    s = Scheduler(ex, max_batch=2)
    consumed = []
    s.cancel(5)                                   # cancelled before it arrives

    def consume(r):
        consumed.append(r.rid)

    orig_launch = ex.launch

    def launch(rs):
        h = orig_launch(rs)
        if [r.rid for r in rs] == [0, 1]:
            s.cancel(4)                           # still queued
        if [r.rid for r in rs] == [2, 3]:
            s.cancel(3)                           # in flight
        return h

    ex.launch = launch
    s.run(reqs, realtime=False, consume=consume)
    _check_terminal(s, reqs, ex)
    st = {r.rid: r.status for r in reqs}
    assert st == {0: "ok", 1: "ok", 2: "ok", 3: "cancelled", 4: "cancelled", 5: "cancelled"}
    assert 4 not in [i for b in ex.launched for i in b] and 5 not in [i for b in ex.launched for i in b]
    assert [2, 3] in ex.launched
    assert ex.discarded == ["result-3"]
    assert sorted(consumed) == [0, 1, 2]
    assert reqs[3].result == {"info": reqs[3].result["info"]}


def test_launch_failure_fails_only_that_batch():
    ex = FakeExecutor(slots=2, launch_fail=lambda rs: any(r.rid == 7 for r in rs))
    reqs = _reqs(20)
    s = Scheduler(ex, max_batch=4)
    s.run(reqs, realtime=False)
    _check_terminal(s, reqs, ex)
    bad = [r for r in reqs if r.status == "error"]
    assert sorted(r.rid for r in bad) == [4, 5, 6, 7]
    assert all("injected launch failure" in r.error for r in bad)
    assert all(r.status == "ok" for r in reqs if r.rid not in (4, 5, 6, 7))
    rec = [b for b in s.batches if "error" in b]
    assert len(rec) == 1 and rec[0]["status"] == {"error": 4}


def test_device_error_at_completion_fails_the_batch():
    """A batch whose results report a device-side error (the workspace error word of a
    timed-out wait, say) ends in "error"; later batches are served."""
    ex = FakeExecutor(slots=2, batch_fail=lambda rs: rs[0].rid == 0)
    reqs = _reqs(9)
    s = Scheduler(ex, max_batch=3)
    s.run(reqs, realtime=False)
    _check_terminal(s, reqs, ex)
    assert [r.status for r in reqs] == ["error"] * 3 + ["ok"] * 6
    assert "ETIMEOUT" in reqs[0].error


def test_queue_limit_rejects_on_arrival():
    """Burst of 30 arrivals at once against a queue of 5 and one slow slot: the
    overflow is rejected immediately, the rest is served."""
    ex = FakeExecutor(slots=1, delay=lambda rs: 0.02)
    reqs = _reqs(30)
    s = Scheduler(ex, max_batch=2, max_queue=5)
    s.run(reqs, realtime=True)
    _check_terminal(s, reqs, ex)
    rej = [r for r in reqs if r.status == "rejected"]
    ok = [r for r in reqs if r.status == "ok"]
    assert rej and ok and len(rej) + len(ok) == 30
    assert all(r.done - r.arrival < 0.01 for r in rej)
    assert all(r.error == "queue full" for r in rej)


def test_capacity_status_is_per_request():
    ex = FakeExecutor(slots=1, capacity=lambda r: 150 if r.rid % 2 else 10 ** 6)
    reqs = _reqs(6, nbits=200)
    s = Scheduler(ex, max_batch=6)
    s.run(reqs, realtime=False)
    assert [r.status for r in reqs] == ["ok", "capacity"] * 3
    rec = s.batches[0]
    assert rec["embedded_bits"] == 3 * 200 + 3 * 150
    assert rec["der_bpp"] == pytest.approx(rec["embedded_bits"] / (6 * 64 * 64))


def test_realtime_arrivals_and_injected_delays():
    """Poisson-like arrivals with per-batch delays that grow with the batch: latency is
    at least the injected delay, requests never start before they arrive, and the
    metrics and JSON lines agree with the requests."""
    rng = np.random.default_rng(3)
    reqs = _reqs(60, kinds=("encode", "decode"), side=0, seed=3)
    t = np.cumsum(rng.exponential(0.002, size=60))
    for r, a in zip(reqs, t):
        r.arrival = float(a)
    starts = {}

    class Stamp(FakeExecutor):
        def launch(self, rs):
            for r in rs:
                starts[r.rid] = s.now()
            return super().launch(rs)

    ex = Stamp(slots=2, delay=lambda rs: 0.001 + 0.0002 * len(rs))
    s = Scheduler(ex, max_batch=8)
    s.run(reqs, realtime=True)
    _check_terminal(s, reqs, ex)
    for r in reqs:
        assert starts[r.rid] >= r.arrival - 1e-9
        assert r.done - starts[r.rid] >= 0.001
    m = s.metrics()
    assert m["requests"] == 60 and m["status"]["ok"] == 60 and m["batches"] == len(ex.launched)
    assert sum(m["latency_hist"]["counts"]) == 60
    assert m["p99_ms"] >= m["p50_ms"] >= 1.0
    lines = [json.loads(x) for x in s.jsonl().splitlines()]
    assert [x["type"] for x in lines] == ["batch"] * len(ex.launched) + ["metrics"]
    assert sum(x["requests"] for x in lines[:-1]) == 60
    assert sum(x["pixels"] for x in lines[:-1]) == sum(r.pixels for r in reqs)


def test_latency_histogram_buckets():
    reqs = _reqs(4)
    for r, lat in zip(reqs, (0.01, 0.06, 1.0, 1e6)):     # ms
        r.arrival, r.done, r.status = 0.0, lat / 1e3, "ok"
    s = Scheduler(FakeExecutor())
    s.completed = reqs
    h = s.metrics()["latency_hist"]
    assert h["upper_edges_ms"] == LAT_EDGES_MS
    c = h["counts"]
    assert c[0] == 1 and c[1] == 1 and c[5] == 1 and c[-1] == 1     # 1.0 ms <= 0.05 * 2^5
    assert latency_stats(reqs + [Request(rid=9, kind="encode", params=None, image=np.zeros((2, 2)),
                                         status="rejected", done=0.5)])["requests"] == 4


def test_idle_wait_does_not_spin():
    """Two requests 50 ms apart: the scheduler sleeps between them (bounded CPU time)."""
    reqs = _reqs(2, spacing=0.05)
    ex = FakeExecutor(slots=1)
    s = Scheduler(ex)
    c0 = time.process_time()
    s.run(reqs, realtime=True)
    assert time.process_time() - c0 < 0.04
    assert all(r.status == "ok" for r in reqs)


def test_admission_window_batches_arrivals_while_busy():
    """With an admission window, requests that arrive while a batch is on the device wait
    (up to the window) and leave together; an idle device takes a request at once."""
    ex = FakeExecutor(slots=2, delay=lambda reqs: 0.02)
    reqs = _reqs(12, spacing=0.001)
    s = Scheduler(ex, max_batch=16, admit_window_ms=8.0)
    s.run(reqs, realtime=True)
    _check_terminal(s, reqs, ex)
    assert ex.launched[0] == [0]                      # the idle device took the first request alone
    assert max(len(b) for b in ex.launched) >= 4
    assert len(ex.launched) <= 5
    # no window: a free slot takes whatever is queued
    ex2 = FakeExecutor(slots=2, delay=lambda reqs: 0.02)
    s2 = Scheduler(ex2, max_batch=16)
    s2.run(_reqs(12, spacing=0.001), realtime=True)
    assert len(ex2.launched) >= len(ex.launched)


def test_held_state_counts_against_the_budget():
    """Device-resident state of earlier requests (reported by the executor) shrinks the
    admission budget: with the budget almost all held, one request runs at a time."""
    reqs = _reqs(6)
    one = reqs[0].device_bytes()

    class Holding(FakeExecutor):
        def state_bytes(self):
            return 10 * one

    ex = Holding(slots=4)
    s = Scheduler(ex, budget_bytes=11.5 * one, max_batch=8)
    s.run(reqs, realtime=False)
    _check_terminal(s, reqs, ex)
    assert ex.max_live == 1 and all(len(b) == 1 for b in ex.launched)
