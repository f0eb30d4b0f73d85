"""Tikhonov-regularised CG-SENSE, (E^H E + lambda I) x = E^H y, on the GPU
against the oracle: every kernel variant in both CG modes, a change of
lambda on the same plan (captured graphs and frame tables rebuilt), centred
k-space, and a batch with a different lambda per instance (bit-identical to
each instance solved alone)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1807_11830_gb300 import sense, synth
from tests.gpu_util import CG_TOL, c64, ensure_built, i32, rel

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _as32(a):
    return np.asarray(a).astype(np.complex64).astype(np.complex128)


def _problem(shape, seed, centred=False):
    ny, nx, C, L, F = shape
    rng = synth.rng_for(seed)
    S = synth.sensitivities(C, ny, nx)
    lines = synth.mask_lines(ny, L, min(4, L), F, rng)
    if centred:
        lines = synth.centred_lines(lines, ny)
    x = synth.random_complex((F, ny, nx), rng)
    y = oracle.forward(_as32(x), _as32(S), lines, centred=centred) + synth.complex_noise((F, C, L, nx), 0.05, rng)
    return S, lines, y


def _solve(plan, y, S, lines, K, tol=0.0):
    F, ny, nx = plan.shape["frames"], plan.shape["ny"], plan.shape["nx"]
    x = torch.empty((F, ny, nx), dtype=torch.complex64, device=DEV)
    it = torch.zeros(F, dtype=torch.int32, device=DEV)
    oc = torch.zeros(F, dtype=torch.int32, device=DEV)
    sense.sense_cg_solve(plan, c64(y), c64(S), i32(lines), K, tol, x, it, None, oc)
    sense.sense_plan_check(plan)
    return x.cpu().numpy(), it.cpu().numpy(), oc.cpu().numpy()


@pytest.mark.parametrize("shape", [(64, 64, 4, 16, 2), (256, 96, 6, 48, 2), (192, 20, 3, 40, 1)],
                         ids=lambda s: "%dx%d" % s[:2])
def test_regularised_cg_every_variant_both_modes(shape):
    ny, nx, C, L, F = shape
    S, lines, y = _problem(shape, 11000 + sum(shape))
    K, lam = 10, 0.0625
    xo, io, _, so = oracle.cg(_as32(y), _as32(S), lines, K, lam=lam)
    plan = sense.Plan(ny, nx, C, F, L)
    sense.sense_plan_set_lambda(plan, lam)
    for v in range(sense.NORM_VARIANTS):
        try:
            sense.sense_plan_set_variant(plan, v)
        except sense.SenseError:
            continue
        for mode in (sense.CG_MODE_GRAPH, sense.CG_MODE_PERSISTENT, sense.CG_MODE_DIRECT):
            sense.sense_plan_set_cg_mode(plan, mode)
            xg, ig, og = _solve(plan, y, S, lines, K)
            assert rel(xg, xo) <= CG_TOL, (v, mode)
            np.testing.assert_array_equal(ig, io)
            np.testing.assert_array_equal(og, so)


def test_lambda_change_on_one_plan_and_tolerance():
    shape = (128, 128, 5, 32, 2)
    ny, nx, C, L, F = shape
    S, lines, y = _problem(shape, 11500)
    plan = sense.Plan(ny, nx, C, F, L)
    for mode in (sense.CG_MODE_GRAPH, sense.CG_MODE_PERSISTENT):
        sense.sense_plan_set_cg_mode(plan, mode)
        for lam in (0.0, 0.25, 4.0, 0.0):  # the same plan, graphs and frame tables rebuilt each time
            sense.sense_plan_set_lambda(plan, lam)
            xg, ig, _ = _solve(plan, y, S, lines, 8)
            assert rel(xg, oracle.cg(_as32(y), _as32(S), lines, 8, lam=lam)[0]) <= CG_TOL, (mode, lam)
        # with a tolerance: regularisation makes the system well conditioned, CG converges
        sense.sense_plan_set_lambda(plan, 0.5)
        xg, ig, og = _solve(plan, y, S, lines, 200, 1e-5)
        xo, io, _, so = oracle.cg(_as32(y), _as32(S), lines, 200, 1e-5, lam=0.5)
        assert np.all(og == sense.CG_CONVERGED) and np.all(so == sense.CG_CONVERGED)
        assert np.all(np.abs(ig.astype(int) - io.astype(int)) <= 1)
        assert rel(xg, xo) <= 10 * CG_TOL
    with pytest.raises(sense.SenseError):
        sense.sense_plan_set_lambda(plan, -1.0)
    with pytest.raises(sense.SenseError):
        sense.sense_plan_set_lambda(plan, float("nan"))


def test_regularised_centred():
    shape = (96, 160, 4, 30, 2)
    ny, nx, C, L, F = shape
    S, lines, y = _problem(shape, 11600, centred=True)
    plan = sense.Plan(ny, nx, C, F, L, centred=True)
    sense.sense_plan_set_lambda(plan, 0.125)
    xg, ig, _ = _solve(plan, y, S, lines, 9)
    assert rel(xg, oracle.cg(_as32(y), _as32(S), lines, 9, centred=True, lam=0.125)[0]) <= CG_TOL


def test_batch_per_instance_lambda():
    specs = [((64, 64, 4, 16, 2), 0.0), ((64, 64, 3, 20, 1), 0.25), ((128, 96, 5, 40, 2), 2.0)]
    inst = [(shape, lam) + _problem(shape, 11700 + k) for k, (shape, lam) in enumerate(specs)]
    shapes = [dict(ny=s[0], nx=s[1], coils=s[2], frames=s[4], lines=s[3]) for s, _, _, _, _ in inst]
    batch = sense.Batch(shapes)
    for k, (_, lam, _, _, _) in enumerate(inst):
        sense.sense_batch_set_lambda(batch, k, lam)
    items = [dict(y=c64(y), S=c64(S), lines=i32(lines),
                  x_out=torch.empty((s[4], s[0], s[1]), dtype=torch.complex64, device=DEV))
             for s, _, S, lines, y in inst]
    K = 7
    sense.sense_batch_cg_solve(batch, items, K)
    sense.sense_batch_check(batch)
    torch.cuda.synchronize()
    for k, (shape, lam, S, lines, y) in enumerate(inst):
        ny, nx, C, L, F = shape
        xb = items[k]["x_out"].cpu().numpy()
        assert rel(xb, oracle.cg(_as32(y), _as32(S), lines, K, lam=lam)[0]) <= CG_TOL, k
        plan = sense.Plan(ny, nx, C, F, L)
        sense.sense_plan_set_lambda(plan, lam)
        sense.sense_plan_set_cg_mode(plan, sense.CG_MODE_PERSISTENT)
        xa, _, _ = _solve(plan, y, S, lines, K)
        np.testing.assert_array_equal(xa, xb)
    batch.close()
