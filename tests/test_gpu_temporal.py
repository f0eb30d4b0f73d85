"""Temporally regularised CG-SENSE on the GPU: the frames of a cine series
coupled into one CG on (E^H E + lambda I + lambda_t L) x = E^H y (L the
cyclic second difference across frames), against the oracle's coupled CG:
every kernel variant, any CG-mode setting (the coupled solve always runs in
the persistent kernel), a tolerance stop on the series residual, centred
k-space, and a batch mixing coupled and independent instances."""
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


def _cine(shape, seed, centred=False):
    ny, nx, C, L, F = shape
    rng = synth.rng_for(seed)
    S = synth.sensitivities(C, ny, nx)
    x = synth.phantom(ny, nx, 8, rng, frames=F, period=F)
    lines = synth.mask_lines(ny, L, min(8, L), F, rng)
    if centred:
        lines = synth.centred_lines(lines, ny)
    y = oracle.forward(_as32(x), _as32(S), lines, centred=centred) + synth.complex_noise((F, C, L, nx), 0.02, rng)
    return S, lines, y


def _solve(plan, y, S, lines, K, tol=0.0):
    F, ny, nx = plan.shape["frames"], plan.shape["ny"], plan.shape["nx"]
    x = torch.empty((F, ny, nx), dtype=torch.complex64, device=DEV)
    it = torch.zeros(F, dtype=torch.int32, device=DEV)
    rr = torch.zeros(F, dtype=torch.float64, device=DEV)
    oc = torch.zeros(F, dtype=torch.int32, device=DEV)
    sense.sense_cg_solve(plan, c64(y), c64(S), i32(lines), K, tol, x, it, rr, oc)
    sense.sense_plan_check(plan)
    return x.cpu().numpy(), it.cpu().numpy(), rr.cpu().numpy(), oc.cpu().numpy()


@pytest.mark.parametrize("shape", [(64, 64, 4, 16, 6), (256, 96, 5, 48, 4), (128, 20, 3, 32, 3)],
                         ids=lambda s: "%dx%d_f%d" % (s[0], s[1], s[4]))
def test_temporal_cg_every_variant(shape):
    ny, nx, C, L, F = shape
    S, lines, y = _cine(shape, 12000 + sum(shape))
    K, lam, lam_t = 10, 0.03125, 0.5
    xo, io, ro, so = oracle.cg(_as32(y), _as32(S), lines, K, lam=lam, lam_t=lam_t)
    plan = sense.Plan(ny, nx, C, F, L)
    sense.sense_plan_set_lambda(plan, lam)
    sense.sense_plan_set_temporal(plan, lam_t)
    for v in range(sense.NORM_VARIANTS):
        try:
            sense.sense_plan_set_variant(plan, v)
        except sense.SenseError:
            continue
        for mode in (sense.CG_MODE_PERSISTENT, sense.CG_MODE_GRAPH):
            sense.sense_plan_set_cg_mode(plan, mode)
            xg, ig, rg, og = _solve(plan, y, S, lines, K)
            assert rel(xg, xo) <= CG_TOL, (v, mode)
            np.testing.assert_array_equal(ig, io)
            np.testing.assert_array_equal(og, so)
            assert np.all(ig == ig[0]) and np.all(rg == rg[0])
            assert np.allclose(rg, ro, rtol=1e-3)
    # the coupling matters: independent frames give a different image
    assert rel(oracle.cg(_as32(y), _as32(S), lines, K, lam=lam)[0], xo) > 10 * CG_TOL


def test_temporal_cg_tolerance_and_weight_changes():
    shape = (96, 96, 4, 24, 5)
    ny, nx, C, L, F = shape
    S, lines, y = _cine(shape, 12500)
    plan = sense.Plan(ny, nx, C, F, L)
    for lam_t in (2.0, 0.0, 0.25):  # the same plan: frame tables rebuilt each time
        sense.sense_plan_set_temporal(plan, lam_t)
        sense.sense_plan_set_lambda(plan, 0.0625)
        xg, ig, rg, og = _solve(plan, y, S, lines, 300, 1e-5)
        xo, io, ro, so = oracle.cg(_as32(y), _as32(S), lines, 300, 1e-5, lam=0.0625, lam_t=lam_t)
        assert np.all(og == sense.CG_CONVERGED) and np.all(so == sense.CG_CONVERGED), lam_t
        assert np.all(np.abs(ig.astype(int) - io.astype(int)) <= 1), (lam_t, ig, io)
        assert np.all(rg <= 1e-5)
        assert rel(xg, xo) <= 10 * CG_TOL, lam_t
    with pytest.raises(sense.SenseError):
        sense.sense_plan_set_temporal(plan, -0.5)


def test_temporal_centred():
    shape = (64, 128, 3, 20, 4)
    ny, nx, C, L, F = shape
    S, lines, y = _cine(shape, 12600, centred=True)
    plan = sense.Plan(ny, nx, C, F, L, centred=True)
    sense.sense_plan_set_temporal(plan, 1.0)
    xg, _, _, _ = _solve(plan, y, S, lines, 8)
    assert rel(xg, oracle.cg(_as32(y), _as32(S), lines, 8, centred=True, lam_t=1.0)[0]) <= CG_TOL


def test_batch_mixes_coupled_and_independent():
    specs = [((64, 64, 4, 16, 4), 0.5), ((64, 64, 3, 20, 2), 0.0), ((128, 96, 4, 32, 3), 2.0)]
    inst = [(shape, lt) + _cine(shape, 12700 + k) for k, (shape, lt) in enumerate(specs)]
    shapes = [dict(ny=s[0], nx=s[1], coils=s[2], frames=s[4], lines=s[3]) for s, _, _, _, _ in inst]
    batch = sense.Batch(shapes)
    for k, (_, lt, _, _, _) in enumerate(inst):
        sense.sense_batch_set_temporal(batch, k, lt)
    items = [dict(y=c64(y), S=c64(S), lines=i32(lines),
                  x_out=torch.empty((s[4], s[0], s[1]), dtype=torch.complex64, device=DEV),
                  iters_out=torch.zeros(s[4], dtype=torch.int32, device=DEV))
             for s, _, S, lines, y in inst]
    K = 7
    sense.sense_batch_cg_solve(batch, items, K)
    sense.sense_batch_check(batch)
    torch.cuda.synchronize()
    for k, (shape, lt, S, lines, y) in enumerate(inst):
        ny, nx, C, L, F = shape
        xb = items[k]["x_out"].cpu().numpy()
        assert rel(xb, oracle.cg(_as32(y), _as32(S), lines, K, lam_t=lt)[0]) <= CG_TOL, k
        plan = sense.Plan(ny, nx, C, F, L)
        sense.sense_plan_set_temporal(plan, lt)
        sense.sense_plan_set_cg_mode(plan, sense.CG_MODE_PERSISTENT)
        xa, _, _, _ = _solve(plan, y, S, lines, K)
        np.testing.assert_array_equal(xa, xb)
    batch.close()
