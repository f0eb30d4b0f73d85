"""The persistent CG kernel's item order changes no arithmetic (GPU).

Every work item computes its own tile or chunk, and the last arriver of a
phase sums the FP64 partials in tile order, so the iteration-major order,
the automatic stagger and any pinned stagger must give the same bits: x, the
iteration counts, the residuals and the outcomes.  The order is pinned
through the test hook declared in include/sense_testing.h.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1807_11830_gb300 import sense, synth
from tests.gpu_util import CG_TOL, c64, ensure_built, i32, make_plan, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _set_order(plan, order):
    lib = sense.load_library()
    lib.sense_testing_plan_set_order.restype = ctypes.c_int
    lib.sense_testing_plan_set_order.argtypes = [ctypes.c_void_p, ctypes.c_int]
    return lib.sense_testing_plan_set_order(plan.handle, order)


def _solve(plan, y, S, lines, iters):
    F, C, L, nx = y.shape
    ny = S.shape[1]
    x = torch.empty((F, ny, nx), dtype=torch.complex64, device="cuda:0")
    it = torch.zeros(F, dtype=torch.int32, device="cuda:0")
    rr = torch.zeros(F, dtype=torch.float64, device="cuda:0")
    oc = torch.zeros(F, dtype=torch.int32, device="cuda:0")
    sense.sense_cg_solve(plan, c64(y), c64(S), i32(lines), iters, 0.0, x, it, rr, oc)
    sense.sense_plan_check(plan)
    return x.cpu().numpy(), it.cpu().numpy(), rr.cpu().numpy(), oc.cpu().numpy()


@pytest.mark.parametrize("variant", [0, 1, 2, 3], ids=lambda v: "v%d" % v)
def test_every_item_order_gives_the_same_bits(variant):
    p = synth.cine_256(frames=6)
    y = oracle.forward(p.x_true, p.S, p.lines) + p.noise
    K = 8
    plan = make_plan(p.S, p.lines)
    sense.sense_plan_set_variant(plan, variant)
    sense.sense_plan_set_cg_mode(plan, sense.CG_MODE_PERSISTENT)
    results = {}
    for order in (-1, -2, 0, 2, 5):
        assert _set_order(plan, order) == sense.SENSE_OK
        results[order] = _solve(plan, y, p.S, p.lines, K)
    ref = results[-1]
    for order, res in results.items():
        for a, b in zip(res, ref):
            np.testing.assert_array_equal(a, b, err_msg="order %d" % order)
    xo, io, _, _ = oracle.cg(y.astype(np.complex64).astype(np.complex128),
                             p.S.astype(np.complex64).astype(np.complex128), p.lines, K)
    assert rel(ref[0].astype(np.complex128), xo) <= CG_TOL
    np.testing.assert_array_equal(ref[1], io)


def test_stagger_must_be_below_the_frame_count():
    p = synth.cine_256(frames=3)
    y = oracle.forward(p.x_true, p.S, p.lines)
    plan = make_plan(p.S, p.lines)
    sense.sense_plan_set_cg_mode(plan, sense.CG_MODE_PERSISTENT)
    assert _set_order(plan, -3) == 1  # SENSE_EINVAL
    assert _set_order(plan, 3) == sense.SENSE_OK  # accepted here; the launch rejects D >= frames
    with pytest.raises(sense.SenseError):
        _solve(plan, y, p.S, p.lines, 2)
    assert _set_order(plan, 2) == sense.SENSE_OK
    _solve(plan, y, p.S, p.lines, 2)
