"""Scheduler logic of the serving queue, on the CPU (fake-device mode: no GPU
work; every frame stops after min(max_iter, fake_iters) ticks).

Covers arrival-order admission, the live-request limit, admission by the
memory budget, refusal of requests that can never fit, cancellation of
pending and running requests, waits with a timeout and unknown ids.
"""
import time

import numpy as np
import pytest

from paper_1807_11830_gb300 import build as sense_build
from paper_1807_11830_gb300 import sense


@pytest.fixture(scope="module", autouse=True)
def _built():
    sense_build.build()
    sense.load_library()


def _req(n=64, coils=4, frames=2, lines=16):
    shape = dict(ny=n, nx=n, coils=coils, frames=frames, lines=lines)
    y = np.zeros((frames, coils, lines, n), np.complex64)
    S = np.zeros((coils, n, n), np.complex64)
    ln = np.tile(np.arange(lines, dtype=np.int32), (frames, 1))
    return shape, y, S, ln


def test_all_requests_complete_in_order_with_one_live():
    q = sense.Queue(fake_device=True, fake_tick_us=200, fake_iters=3, max_live=1)
    ids = [q.submit(*_req(), max_iter=10) for _ in range(6)]
    done_order = []
    pending = set(ids)
    while pending:
        for rid in list(pending):
            st, _ = q.poll(rid)
            if st == sense.REQ_DONE:
                done_order.append(rid)
                pending.discard(rid)
        time.sleep(0.001)
    assert done_order == ids  # one live request at a time: strict arrival order
    for rid in ids:
        it = np.zeros(2, np.int32)
        oc = np.zeros(2, np.int32)
        q.wait(rid, iters=it, outcome=oc)
        assert list(it) == [3, 3] and list(oc) == [sense.CG_CONVERGED] * 2
    st = q.stats()
    assert st["completed"] == 6 and st["admitted"] == 6 and st["ticks"] >= 18
    assert st["p99_ms"] >= st["p50_ms"] > 0
    q.close()


def test_iteration_level_batching_runs_requests_together():
    q = sense.Queue(fake_device=True, fake_tick_us=2000, fake_iters=20)
    ids = [q.submit(*_req(), max_iter=20) for _ in range(5)]
    peak = 0
    for _ in range(50):
        peak = max(peak, q.stats()["live"])
        time.sleep(0.001)
    assert peak >= 2  # several requests advance in the same ticks
    for rid in ids:
        q.wait(rid)
    st = q.stats()
    assert st["ticks"] < 5 * 20  # far fewer ticks than a serial loop would need
    q.close()


def test_budget_admission_and_refusal():
    shape, y, S, ln = _req()
    # find one request's need by a budget that refuses it
    q = sense.Queue(fake_device=True, hbm_budget_bytes=1024)
    with pytest.raises(sense.SenseError) as ei:
        q.submit(shape, y, S, ln, max_iter=5)
    assert ei.value.status == 7  # SENSE_EQUEUE_FULL
    assert q.stats()["refused"] == 1
    q.close()
    # the exact need of one request, by bisection on the refusal boundary
    lo, hi = 1024, 1 << 30  # refused at lo, accepted at hi
    while hi - lo > 1:
        mid = (lo + hi) // 2
        qq = sense.Queue(fake_device=True, hbm_budget_bytes=mid)
        try:
            qq.submit(shape, y, S, ln, max_iter=1)
            hi = mid
        except sense.SenseError:
            lo = mid
        qq.close()
    need = hi
    q = sense.Queue(fake_device=True, hbm_budget_bytes=2 * need + need // 2, fake_tick_us=500, fake_iters=10)
    ids = [q.submit(shape, y, S, ln, max_iter=10) for _ in range(6)]
    peak = 0
    for _ in range(400):
        st = q.stats()
        peak = max(peak, st["live"])
        assert st["hbm_in_use"] <= st["hbm_budget"]
        if st["completed"] == 6:
            break
        time.sleep(0.001)
    for rid in ids:
        q.wait(rid)
    assert peak == 2  # two fit the budget, the third waits for one to retire
    q.close()


def test_cancel_pending_and_running():
    q = sense.Queue(fake_device=True, fake_tick_us=1000, fake_iters=50, max_live=1)
    a = q.submit(*_req(), max_iter=50)
    b = q.submit(*_req(), max_iter=50)
    time.sleep(0.01)
    assert q.poll(a)[0] == sense.REQ_RUNNING and q.poll(b)[0] == sense.REQ_PENDING
    q.cancel(b)
    q.cancel(a)
    with pytest.raises(sense.SenseError):
        q.wait(a)
    with pytest.raises(sense.SenseError):
        q.wait(b)
    c = q.submit(*_req(), max_iter=2)
    q.wait(c)
    st = q.stats()
    assert st["cancelled"] == 2 and st["completed"] == 1
    q.close()


def test_unknown_ids_and_wait_timeout():
    q = sense.Queue(fake_device=True, fake_tick_us=2000, fake_iters=100)
    with pytest.raises(sense.SenseError) as ei:
        q.poll(12345)
    assert ei.value.status == 8
    rid = q.submit(*_req(), max_iter=100)
    with pytest.raises(sense.SenseError) as ei:
        q.wait(rid, timeout_s=0.01)
    assert ei.value.status == 5
    q.cancel(rid)
    q.close()


def test_bad_submissions():
    q = sense.Queue(fake_device=True)
    shape, y, S, ln = _req()
    bad = dict(shape, ny=100, nx=100)
    with pytest.raises(sense.SenseError) as ei:
        q.submit(bad, y, S, ln, max_iter=3)
    assert ei.value.status == 2
    with pytest.raises(sense.SenseError):
        q.submit(shape, y, S, ln, max_iter=0)
    q.close()


def test_injected_admission_failures_release_their_budget():
    # every third admission fails as if a device allocation had failed
    q = sense.Queue(fake_device=True, fake_tick_us=200, fake_iters=2, max_live=1, fail_admit_every=3)
    ids = [q.submit(*_req(), max_iter=5) for _ in range(7)]
    failed = []
    for k, rid in enumerate(ids):
        try:
            q.wait(rid)
        except sense.SenseError as e:
            assert e.status == 3 and "injected" in str(e)  # SENSE_ENOMEM
            failed.append(k)
    assert failed == [2, 5]  # admissions 3 and 6 in arrival order
    st = q.stats()
    assert st["failed"] == 2 and st["completed"] == 5 and st["admitted"] == 7
    assert st["hbm_in_use"] == 0 and st["live"] == 0
    q.close()
    with pytest.raises(sense.SenseError) as ei:
        sense.Queue(fake_device=True, fail_admit_every=-1)
    assert ei.value.status == 1


def test_request_log_records_every_request(tmp_path, monkeypatch):
    import json

    log = tmp_path / "requests.jsonl"
    monkeypatch.setenv("SENSE_QUEUE_LOG", str(log))
    q = sense.Queue(fake_device=True, fake_tick_us=1000, fake_iters=3, max_live=1, fail_admit_every=2)
    a = q.submit(*_req(n=64, frames=2), max_iter=10)
    b = q.submit(*_req(n=32, frames=1), max_iter=10)  # second admission: injected failure
    c = q.submit(*_req(n=64, frames=3), max_iter=10)
    d = q.submit(*_req(), max_iter=10)
    q.cancel(d)  # still pending behind a and c (one live at a time)
    q.wait(a)
    with pytest.raises(sense.SenseError):
        q.wait(b)
    q.wait(c)
    with pytest.raises(sense.SenseError):
        q.wait(d)
    q.close()
    recs = {r["id"]: r for r in map(json.loads, log.read_text().splitlines())}
    assert set(recs) == {a, b, c, d}
    ra, rb, rc, rd = recs[a], recs[b], recs[c], recs[d]
    assert (ra["state"], rb["state"], rc["state"], rd["state"]) == ("done", "failed", "done", "cancelled")
    assert rb["status"] == 3 and ra["status"] == 0
    assert (ra["ny"], ra["frames"], rb["ny"], rc["frames"]) == (64, 2, 32, 3)
    for r in (ra, rc):
        assert r["submit_ms"] <= r["admit_ms"] <= r["first_tick_ms"] <= r["done_ms"]
        assert abs(r["latency_ms"] - (r["done_ms"] - r["submit_ms"])) < 1e-2
        assert r["ticks"] == 3 and r["iters"] == 3 and r["max_rel_resid"] == 0.0 and r["max_iter"] == 10
    assert "first_tick_ms" not in rb and "admit_ms" in rb and "iters" not in rb
    assert "admit_ms" not in rd and "first_tick_ms" not in rd
    assert rc["admit_ms"] >= ra["done_ms"] - 1e-3  # one live at a time: c is admitted after a retires


MiB = 1 << 20


def test_staging_arena_reuses_space_across_shapes():
    q = sense.Queue(fake_device=True, fake_tick_us=100, fake_iters=1)
    shapes = [dict(n=64, coils=4, frames=2, lines=16), dict(n=128, coils=8, frames=3, lines=40),
              dict(n=96, coils=6, frames=1, lines=30)]
    for rep in range(3):
        for sp in shapes:
            q.wait(q.submit(*_req(**sp), max_iter=2))
        st = q.stats()
        assert st["staging_in_use"] == 0  # everything returned after the waits
        assert st["staging_reserved"] == 256 * MiB  # one chunk serves every shape, every time
    # several requests held at once still share the one chunk, and their space coalesces back
    ids = [q.submit(*_req(**sp), max_iter=2) for sp in shapes * 3]
    assert q.stats()["staging_in_use"] > 0
    for rid in ids[1::2] + ids[0::2]:  # out of order
        q.wait(rid)
    st = q.stats()
    assert st["staging_in_use"] == 0 and st["staging_reserved"] == 256 * MiB
    q.close()


def test_staging_arena_large_request_gets_its_own_chunk():
    q = sense.Queue(fake_device=True, fake_tick_us=100, fake_iters=1)
    big = dict(n=384, coils=8, frames=8, lines=384)  # y: 8*8*384*384*8 B = 72 MiB, well under a chunk
    q.wait(q.submit(*_req(**big), max_iter=2))
    assert q.stats()["staging_reserved"] == 256 * MiB
    huge = dict(n=384, coils=30, frames=8, lines=384)  # y: 270 MiB, more than a chunk
    q.wait(q.submit(*_req(**huge), max_iter=2))
    st = q.stats()
    assert st["staging_reserved"] == 256 * MiB + 270 * MiB and st["staging_in_use"] == 0
    # the freed large chunk is reused, no third chunk
    reserved = st["staging_reserved"]
    q.wait(q.submit(*_req(**huge), max_iter=2))
    assert q.stats()["staging_reserved"] == reserved
    q.close()


def test_staging_reservation_and_growth():
    q = sense.Queue(fake_device=True, fake_tick_us=2000, fake_iters=100, max_live=1,
                    staging_reserve_bytes=300 * MiB)
    assert q.stats()["staging_reserved"] == 300 * MiB
    # requests held at once beyond the reservation: chunks grow with what is reserved
    big = dict(n=384, coils=16, frames=8, lines=384)  # y: 144 MiB
    ids = [q.submit(*_req(**big), max_iter=100) for _ in range(4)]
    st = q.stats()
    assert st["staging_in_use"] >= 4 * 144 * MiB and st["staging_reserved"] >= st["staging_in_use"]
    assert st["staging_reserved"] < 2 * st["staging_in_use"] + 300 * MiB  # growth stays proportionate
    for rid in ids:
        q.cancel(rid)
    for rid in ids:
        with pytest.raises(sense.SenseError):
            q.wait(rid)
    assert q.stats()["staging_in_use"] == 0
    q.close()


def test_set_variant_before_first_request():
    q = sense.Queue(fake_device=True, fake_tick_us=100, fake_iters=1)
    assert q.variant(64, 64) == -1
    q.set_variant(256, 256, 1)
    assert q.variant(256, 256) == 1
    q.set_variant(256, 256, 1)  # the same again is fine
    with pytest.raises(sense.SenseError) as ei:
        q.set_variant(256, 256, 2)  # the class already has one
    assert ei.value.status == 1
    with pytest.raises(sense.SenseError):
        q.set_variant(64, 64, 3)  # 64 has no variant 3
    with pytest.raises(sense.SenseError) as ei:
        q.set_variant(100, 100, 0)
    assert ei.value.status == 2
    q.close()


def test_live_work_cap_admits_in_arrival_order():
    one = 64 * 64 * 4 * 2  # frames x coils x ny x nx of _req()
    q = sense.Queue(fake_device=True, fake_tick_us=1000, fake_iters=5, max_live_work=2 * one)
    ids = [q.submit(*_req(), max_iter=5) for _ in range(6)]
    peak, order, pending = 0, [], set(ids)
    while pending:
        peak = max(peak, q.stats()["live"])
        for rid in sorted(pending):
            if q.poll(rid)[0] == sense.REQ_DONE:
                order.append(rid)
                pending.discard(rid)
        time.sleep(0.0002)
    assert peak == 2 and order == ids
    for rid in ids:
        q.wait(rid)
    q.close()
    # a request larger than the cap still runs, alone
    q = sense.Queue(fake_device=True, fake_tick_us=200, fake_iters=2, max_live_work=one // 2)
    a, b = q.submit(*_req(), max_iter=2), q.submit(*_req(), max_iter=2)
    q.wait(a)
    q.wait(b)
    assert q.stats()["completed"] == 2
    q.close()


def test_saturation_admission_keeps_the_oldest_requests_live():
    """With admit_waves set, requests are admitted in arrival order only while
    the live normal-operator work is below that many device waves (the request
    that crosses it is admitted).  Here each request is 0.026 waves (4 frames x
    2 column tiles over 152 SMs x 2 resident blocks), so a cap of 0.03 keeps at
    most two requests live, and they complete in arrival order."""
    q = sense.Queue(fake_device=True, fake_tick_us=1000, fake_iters=4, admit_waves=0.03)
    ids = [q.submit(*_req(frames=4), max_iter=10) for _ in range(6)]
    peak, done_order, pending = 0, [], set(ids)
    while pending:
        peak = max(peak, q.stats()["live"])
        for rid in list(pending):
            if q.poll(rid)[0] == sense.REQ_DONE:
                done_order.append(rid)
                pending.discard(rid)
        time.sleep(0.0005)
    assert peak == 2
    assert done_order == ids
    for rid in ids:
        q.wait(rid)
    q.close()


def test_saturation_admission_off_admits_everything():
    q = sense.Queue(fake_device=True, fake_tick_us=3000, fake_iters=20, admit_waves=-1.0)
    ids = [q.submit(*_req(frames=4), max_iter=20) for _ in range(6)]
    peak = 0
    for _ in range(40):
        peak = max(peak, q.stats()["live"])
        time.sleep(0.001)
    assert peak == 6
    for rid in ids:
        q.wait(rid)
    q.close()


def test_test_hooks_are_not_part_of_the_public_config():
    """The scheduler's test hooks live in sense_testing.h, not in sense_queue_cfg."""
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    public = open(os.path.join(root, "include", "sense.h")).read()
    i = public.index("typedef struct {\n  size_t hbm_budget_bytes;")
    cfg = public[i:public.index("} sense_queue_cfg;")]
    for hook in ("fake_device", "fake_tick_us", "fake_iters", "fail_admit_every"):
        assert hook not in cfg
    testing = open(os.path.join(root, "include", "sense_testing.h")).read()
    assert "sense_queue_create_with_hooks" in testing and "fail_admit_every" in testing
