"""Serving queue with continuous batching on the GPU.

Requests of different shapes, iteration budgets and tolerances are submitted
while others are running; each result is checked against the FP64 oracle
and against the same problem solved alone by a plan with the queue's kernel
variant for its size class (persistent mode): they must agree bit for bit,
since a frame's iterates do not depend on which other frames share a tick.
"""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_1807_11830_gb300 import sense, synth
from tests.gpu_util import CG_TOL, ensure_built, rel

pytestmark = pytest.mark.gpu

SPECS = [  # n, coils, frames, accel, max_iter, tol, storage
    (64, 4, 2, 3, 8, 0.0, sense.STORE_C64),
    (128, 6, 1, 2, 12, 0.0, sense.STORE_C64),
    (64, 3, 3, 4, 20, 3e-3, sense.STORE_C64),
    (192, 8, 2, 4, 6, 0.0, sense.STORE_C64),
    (128, 5, 2, 3, 10, 0.0, sense.STORE_BF16),
    (64, 4, 1, 2, 15, 0.0, sense.STORE_C64),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _host_inputs(k, spec):
    n, C, F, R, K, tol, storage = spec
    sp = dict(n=n, coils=C, frames=F, accel=R, lines=synth.lines_for_acceleration(n, R), centre=synth.centre_for(n))
    p = synth.mix_instance(sp, 1300 + k)
    y = oracle.forward(p.x_true, p.S, p.lines) + p.noise
    if storage == sense.STORE_BF16:
        yh = oracle.bf16_rne(np.ascontiguousarray(y, np.complex64).view(np.float32)).reshape(y.shape + (2,))
        Sh = oracle.bf16_rne(np.ascontiguousarray(p.S, np.complex64).view(np.float32)).reshape(p.S.shape + (2,))
        yq, Sq = oracle.quantize_c64_bf16(y), oracle.quantize_c64_bf16(p.S)
    else:
        yh, Sh = np.ascontiguousarray(y, np.complex64), np.ascontiguousarray(p.S, np.complex64)
        yq, Sq = yh.astype(np.complex128), Sh.astype(np.complex128)
    shape = dict(ny=n, nx=n, coils=C, frames=F, lines=p.lines.shape[1], storage=storage)
    return shape, yh, Sh, np.ascontiguousarray(p.lines, np.int32), yq, Sq


def test_served_results_equal_alone_and_oracle():
    q = sense.Queue(device=0)
    inputs = [_host_inputs(k, sp) for k, sp in enumerate(SPECS)]
    ids = []
    for k, (shape, yh, Sh, ln, _, _) in enumerate(inputs):
        ids.append(q.submit(shape, yh, Sh, ln, max_iter=SPECS[k][4], rel_tol=SPECS[k][5]))
        if k == 2:
            time.sleep(0.02)  # the rest arrive while the first ones are running
    for k, rid in enumerate(ids):
        shape, yh, Sh, ln, yq, Sq = inputs[k]
        n, C, F, R, K, tol, storage = SPECS[k]
        x = np.empty((F, n, n), np.complex64)
        it = np.empty(F, np.int32)
        rr = np.empty(F, np.float64)
        oc = np.empty(F, np.int32)
        q.wait(rid, x, it, rr, oc)
        # oracle
        xo, io, _, so = oracle.cg(yq, Sq, ln, K, tol)
        assert rel(x.astype(np.complex128), xo) <= CG_TOL, k
        if tol == 0.0:
            np.testing.assert_array_equal(it, io)
            np.testing.assert_array_equal(oc, so)
        # alone, same variant, persistent mode
        plan = sense.Plan(n, n, C, F, shape["lines"], storage)
        sense.sense_plan_set_variant(plan, q.variant(n, n, storage))
        sense.sense_plan_set_cg_mode(plan, sense.CG_MODE_PERSISTENT)
        dev = "cuda:0"
        if storage == sense.STORE_BF16:
            y_d = torch.from_numpy(yh.view(np.int16)).to(dev).view(torch.bfloat16)
            S_d = torch.from_numpy(Sh.view(np.int16)).to(dev).view(torch.bfloat16)
        else:
            y_d, S_d = torch.from_numpy(yh).to(dev), torch.from_numpy(Sh).to(dev)
        xa = torch.empty((F, n, n), dtype=torch.complex64, device=dev)
        ita = torch.zeros(F, dtype=torch.int32, device=dev)
        sense.sense_cg_solve(plan, y_d, S_d, torch.from_numpy(ln).to(dev), K, tol, xa, ita)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(xa.cpu().numpy(), x)
        np.testing.assert_array_equal(ita.cpu().numpy(), it)
    st = q.stats()
    assert st["completed"] == len(SPECS) and st["failed"] == 0
    assert st["ticks"] < sum(sp[4] for sp in SPECS)  # requests shared ticks
    assert st["hbm_in_use"] == 0
    q.close()


def test_queue_budget_holds_requests_back():
    # a budget for about one request at a time: all still complete, one by one
    shape, yh, Sh, ln, _, _ = _host_inputs(0, SPECS[0])
    probe = sense.Queue(device=0, hbm_budget_bytes=1 << 40)
    rid = probe.submit(shape, yh, Sh, ln, max_iter=4)
    probe.wait(rid)
    probe.close()
    lo, hi = 1 << 10, 1 << 32
    while hi - lo > 1:  # the exact need of one request
        mid = (lo + hi) // 2
        qq = sense.Queue(device=0, hbm_budget_bytes=mid, fake_device=True)
        try:
            qq.submit(shape, yh, Sh, ln, max_iter=1)
            hi = mid
        except sense.SenseError:
            lo = mid
        qq.close()
    q = sense.Queue(device=0, hbm_budget_bytes=hi + hi // 2, iters_per_tick=1)
    ids = [q.submit(shape, yh, Sh, ln, max_iter=6) for _ in range(4)]
    for rid in ids:
        q.wait(rid)
    st = q.stats()
    assert st["completed"] == 4 and st["ticks"] >= 4 * 6  # never two at once
    q.close()


def test_large_requests_staged_in_parallel_equal_alone():
    """Inputs of 32 MiB and more are copied into staging by several threads;
    such requests, submitted back to back so their staging coexists in the
    arena, give the same bits as the same problems solved alone."""
    dev = "cuda:0"
    q = sense.Queue(device=0)
    K = 5
    specs = [(256, 24, 8, 128, 3100), (192, 30, 10, 96, 3101), (256, 20, 8, 128, 3102)]
    reqs = []
    for n, C, F, L, seed in specs:
        rng = synth.rng_for(seed)
        S = np.ascontiguousarray(synth.sensitivities(C, n, n), np.complex64)
        lines = np.ascontiguousarray(synth.mask_lines(n, L, synth.centre_for(n), F, rng), np.int32)
        y = np.ascontiguousarray(synth.random_complex((F, C, L, n), rng), np.complex64)
        assert y.nbytes >= 32 << 20
        shape = dict(ny=n, nx=n, coils=C, frames=F, lines=L)
        reqs.append((shape, y, S, lines, q.submit(shape, y, S, lines, max_iter=K)))
    assert q.stats()["staging_reserved"] >= 256 << 20
    for shape, y, S, lines, rid in reqs:
        F, n = shape["frames"], shape["ny"]
        x = np.empty((F, n, n), np.complex64)
        q.wait(rid, x)
        plan = sense.Plan(n, n, shape["coils"], F, shape["lines"])
        sense.sense_plan_set_variant(plan, q.variant(n, n))
        sense.sense_plan_set_cg_mode(plan, sense.CG_MODE_PERSISTENT)
        xa = torch.empty((F, n, n), dtype=torch.complex64, device=dev)
        sense.sense_cg_solve(plan, torch.from_numpy(y).to(dev), torch.from_numpy(S).to(dev),
                             torch.from_numpy(lines).to(dev), K, 0.0, xa)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(xa.cpu().numpy(), x)
    st = q.stats()
    assert st["staging_in_use"] == 0 and st["hbm_in_use"] == 0
    q.close()


def test_pinned_class_variant_is_used():
    """A size class pinned with sense_queue_set_variant runs that variant:
    served results equal a plan solve with it, bit for bit."""
    dev = "cuda:0"
    n, C, F, L, K = 256, 6, 3, 64, 6
    rng = synth.rng_for(3200)
    S = np.ascontiguousarray(synth.sensitivities(C, n, n), np.complex64)
    lines = np.ascontiguousarray(synth.mask_lines(n, L, synth.centre_for(n), F, rng), np.int32)
    y = np.ascontiguousarray(synth.random_complex((F, C, L, n), rng), np.complex64)
    shape = dict(ny=n, nx=n, coils=C, frames=F, lines=L)
    for variant in (1, 3):
        q = sense.Queue(device=0)
        q.set_variant(n, n, variant)
        x = np.empty((F, n, n), np.complex64)
        q.wait(q.submit(shape, y, S, lines, max_iter=K), x)
        assert q.variant(n, n) == variant
        q.close()
        plan = sense.Plan(n, n, C, F, L)
        sense.sense_plan_set_variant(plan, variant)
        sense.sense_plan_set_cg_mode(plan, sense.CG_MODE_PERSISTENT)
        xa = torch.empty((F, n, n), dtype=torch.complex64, device=dev)
        sense.sense_cg_solve(plan, torch.from_numpy(y).to(dev), torch.from_numpy(S).to(dev),
                             torch.from_numpy(lines).to(dev), K, 0.0, xa)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(xa.cpu().numpy(), x)
