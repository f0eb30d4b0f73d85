"""Failure detection on the GPU without a GPU fault.

Non-finite input is the numerical failure a reconstruction service meets
(a corrupted k-space sample, a map with Inf).  CG must stop the affected
frame at once -- outcome breakdown, residual NaN, image zero -- and leave
every other frame bit for bit as it would be without it.  The serving
queue reports such a request with SENSE_ENUMERIC and still returns its
outputs.  Admission failures are injected on the host by the queue's test
hook: the request fails with SENSE_ENOMEM, its partial device allocations
are released, and the requests around it complete with correct results.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1807_11830_gb300 import sense, synth
from tests.gpu_util import CG_TOL, DEV, c64, ensure_built, i32, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _problem(n, C, F, L, seed):
    rng = synth.rng_for(seed)
    S = synth.sensitivities(C, n, n)
    lines = synth.mask_lines(n, L, min(8, L), F, rng)
    x = synth.random_complex((F, n, n), rng)
    y = oracle.forward(x, S, lines) + 1e-3 * synth.random_complex((F, C, L, n), rng)
    return S, lines, y


def _solve(plan, y, S, lines, K, tol=0.0):
    F, n = y.shape[0], S.shape[1]
    x = torch.empty((F, n, n), dtype=torch.complex64, device=DEV)
    it = torch.full((F,), -1, dtype=torch.int32, device=DEV)
    rr = torch.zeros(F, dtype=torch.float64, device=DEV)
    oc = torch.zeros(F, dtype=torch.int32, device=DEV)
    sense.sense_cg_solve(plan, c64(y), c64(S), i32(lines), K, tol, x, it, rr, oc)
    sense.sense_plan_check(plan)
    return x.cpu().numpy(), it.cpu().numpy(), rr.cpu().numpy(), oc.cpu().numpy()


@pytest.mark.parametrize("mode", [sense.CG_MODE_GRAPH, sense.CG_MODE_PERSISTENT])
@pytest.mark.parametrize("tol", [0.0, 1e-3])
@pytest.mark.parametrize("bad", ["nan", "inf"])
def test_nonfinite_frame_stops_alone(mode, tol, bad):
    n, C, F, L, K = 64, 4, 3, 22, 12
    S, lines, y = _problem(n, C, F, L, 2024)
    y_bad = y.copy()
    y_bad[1, 2, 5, 7] = np.nan if bad == "nan" else np.inf
    plan = sense.Plan(n, n, C, F, L)
    sense.sense_plan_set_cg_mode(plan, mode)
    xc, ic, rc, oc = _solve(plan, y, S, lines, K, tol)
    xb, ib, rb, ob = _solve(plan, y_bad, S, lines, K, tol)
    for f in (0, 2):  # the other frames: bit for bit
        np.testing.assert_array_equal(xb[f], xc[f])
        assert ib[f] == ic[f] and ob[f] == oc[f] and rb[f] == rc[f]
    assert ob[1] == sense.CG_BREAKDOWN and ib[1] == 0 and np.isnan(rb[1])
    assert not np.any(xb[1])
    if tol == 0.0:
        xo, io, _, _ = oracle.cg(y.astype(np.complex64).astype(np.complex128), S.astype(np.complex64), lines, K)
        assert rel(xc.astype(np.complex128), xo) <= CG_TOL
        np.testing.assert_array_equal(ic, io)


def test_nonfinite_map_stops_every_frame():
    n, C, F, L, K = 64, 3, 2, 22, 6
    S, lines, y = _problem(n, C, F, L, 2025)
    S_bad = S.copy()
    S_bad[1, 10, 20] = np.inf
    plan = sense.Plan(n, n, C, F, L)
    x, it, rr, oc = _solve(plan, y, S_bad, lines, K)
    assert np.all(oc == sense.CG_BREAKDOWN) and np.all(it == 0) and np.all(np.isnan(rr))
    assert not np.any(x)


def test_nonfinite_instance_in_batch_stops_alone():
    n, C, F, L, K = 64, 4, 2, 22, 8
    probs = [_problem(n, C, F, L, 2030 + k) for k in range(3)]
    probs[1][2][0, 1, 3, 4] = np.nan  # instance 1, frame 0
    shapes = [dict(ny=n, nx=n, coils=C, frames=F, lines=L) for _ in probs]
    batch = sense.Batch(shapes)
    items = []
    for S, lines, y in probs:
        items.append(dict(y=c64(y), S=c64(S), lines=i32(lines),
                          x_out=torch.empty((F, n, n), dtype=torch.complex64, device=DEV),
                          iters_out=torch.zeros(F, dtype=torch.int32, device=DEV),
                          rel_resid_out=torch.zeros(F, dtype=torch.float64, device=DEV),
                          outcome_out=torch.zeros(F, dtype=torch.int32, device=DEV)))
    sense.sense_batch_cg_solve(batch, items, K)
    sense.sense_batch_check(batch)
    torch.cuda.synchronize()
    oc = items[1]["outcome_out"].cpu().numpy()
    assert oc[0] == sense.CG_BREAKDOWN and np.isnan(items[1]["rel_resid_out"].cpu().numpy()[0])
    assert not torch.any(items[1]["x_out"][0] != 0)
    for k in (0, 2):
        S, lines, y = probs[k]
        xo, io, _, so = oracle.cg(y.astype(np.complex64).astype(np.complex128), S.astype(np.complex64), lines, K)
        assert rel(items[k]["x_out"].cpu().numpy().astype(np.complex128), xo) <= CG_TOL
        np.testing.assert_array_equal(items[k]["outcome_out"].cpu().numpy(), so)
    # frame 1 of the bad instance is untouched by its sibling
    S, lines, y = probs[1]
    xo, _, _, _ = oracle.cg(y[1:].astype(np.complex64).astype(np.complex128), S.astype(np.complex64), lines[1:], K)
    assert rel(items[1]["x_out"][1:].cpu().numpy().astype(np.complex128), xo) <= CG_TOL
    batch.close()


def _host(n, C, F, L, seed):
    S, lines, y = _problem(n, C, F, L, seed)
    shape = dict(ny=n, nx=n, coils=C, frames=F, lines=L)
    return shape, np.ascontiguousarray(y, np.complex64), np.ascontiguousarray(S, np.complex64), \
        np.ascontiguousarray(lines, np.int32)


def test_queue_reports_nonfinite_request():
    q = sense.Queue(device=0)
    K = 10
    good = _host(64, 4, 2, 22, 2040)
    bad = _host(64, 4, 2, 22, 2041)
    bad[1][1, 0, 2, 3] = np.nan
    ra = q.submit(*good, max_iter=K)
    rb = q.submit(*bad, max_iter=K)
    x = np.empty((2, 64, 64), np.complex64)
    it = np.empty(2, np.int32)
    rr = np.empty(2, np.float64)
    oc = np.empty(2, np.int32)
    with pytest.raises(sense.SenseError) as ei:
        q.wait(rb, x, it, rr, oc)
    assert ei.value.status == 6  # SENSE_ENUMERIC, outputs still copied
    assert oc[1] == sense.CG_BREAKDOWN and it[1] == 0 and np.isnan(rr[1]) and not np.any(x[1])
    xo, io, _, so = oracle.cg(bad[1][:1].astype(np.complex128), bad[2], bad[3][:1], K)
    assert rel(x[:1].astype(np.complex128), xo) <= CG_TOL and oc[0] == so[0]
    q.wait(ra, x, it, rr, oc)
    xo, io, _, so = oracle.cg(good[1].astype(np.complex128), good[2], good[3], K)
    assert rel(x.astype(np.complex128), xo) <= CG_TOL
    np.testing.assert_array_equal(oc, so)
    q.close()


def test_queue_injected_admission_failure_on_device():
    q = sense.Queue(device=0, fail_admit_every=2)
    K = 8
    reqs = [_host(64 if k % 2 == 0 else 128, 3 + k % 3, 1 + k % 2, 22 if k % 2 == 0 else 43, 2050 + k)
            for k in range(5)]
    ids = [q.submit(*r, max_iter=K) for r in reqs]
    failed = []
    for k, (rid, r) in enumerate(zip(ids, reqs)):
        shape, y, S, lines = r
        x = np.empty((shape["frames"], shape["ny"], shape["nx"]), np.complex64)
        try:
            q.wait(rid, x)
        except sense.SenseError as e:
            assert e.status == 3 and "injected" in str(e)  # SENSE_ENOMEM
            failed.append(k)
            continue
        xo, _, _, _ = oracle.cg(y.astype(np.complex128), S, lines, K)
        assert rel(x.astype(np.complex128), xo) <= CG_TOL, k
    assert failed == [1, 3]
    st = q.stats()
    assert st["failed"] == 2 and st["completed"] == 3 and st["hbm_in_use"] == 0
    q.close()
