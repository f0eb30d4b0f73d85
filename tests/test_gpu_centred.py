"""Centred k-space (DC at n/2) on the GPU against the oracle's centred
transforms (fftshift . F . ifftshift): every operator, CG in both modes and
every kernel variant, BF16 storage, the batch, the serving queue and the
allocation-free adjoint."""
import numpy as np
import pytest
import torch

import oracle
from paper_1807_11830_gb300 import sense, synth
from tests.gpu_util import CG_TOL, OP_TOL, bf16_pairs_from_oracle, c64, ensure_built, i32, rel

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

SHAPES = [  # ny, nx, coils, lines, frames
    (64, 64, 4, 21, 2),
    (256, 96, 3, 64, 1),
    (160, 160, 8, 160, 1),
    (96, 128, 5, 40, 2),
    (256, 20, 2, 64, 2),
    (384, 384, 2, 96, 1),
    (12, 8, 2, 5, 3),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _as32(a):
    return np.asarray(a).astype(np.complex64).astype(np.complex128)


def _problem(shape, seed):
    ny, nx, C, L, F = shape
    rng = synth.rng_for(seed)
    S = synth.sensitivities(C, ny, nx)
    lines = synth.centred_lines(synth.mask_lines(ny, L, min(4, L), F, rng), ny)
    x = synth.random_complex((F, ny, nx), rng)
    y = synth.random_complex((F, C, L, nx), rng)
    return x, S, lines, y


def _plan(S, lines, storage=sense.STORE_C64):
    C, ny, nx = S.shape
    F, L = lines.shape
    return sense.Plan(ny, nx, C, F, L, storage, centred=True)


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "%dx%d_c%d_l%d_f%d" % s)
def test_centred_operators(shape):
    ny, nx, C, L, F = shape
    x, S, lines, y = _problem(shape, 8000 + sum(shape))
    x32, S32, y32 = _as32(x), _as32(S), _as32(y)
    plan = _plan(S, lines)
    # E
    yo = torch.empty((F, C, L, nx), dtype=torch.complex64, device=DEV)
    sense.sense_forward(plan, c64(x), c64(S), i32(lines), yo)
    sense.sense_plan_check(plan)
    assert rel(yo.cpu().numpy(), oracle.forward(x32, S32, lines, centred=True)) <= OP_TOL
    # E^H
    xo = torch.empty((F, ny, nx), dtype=torch.complex64, device=DEV)
    sense.sense_adjoint(plan, c64(y), c64(S), i32(lines), xo)
    sense.sense_plan_check(plan)
    assert rel(xo.cpu().numpy(), oracle.adjoint(y32, S32, lines, centred=True)) <= OP_TOL
    # E^H E, every variant
    expect = oracle.normal(x32, S32, lines, centred=True)
    for v in range(sense.NORM_VARIANTS):
        try:
            sense.sense_plan_set_variant(plan, v)
        except sense.SenseError:
            continue
        qo = torch.empty((F, ny, nx), dtype=torch.complex64, device=DEV)
        sense.sense_normal(plan, c64(x), c64(S), i32(lines), qo)
        sense.sense_plan_check(plan)
        assert rel(qo.cpu().numpy(), expect) <= OP_TOL, v
    # RSS
    ro = torch.empty((F, ny, nx), dtype=torch.float32, device=DEV)
    sense.sense_rss(plan, c64(y), i32(lines), ro)
    sense.sense_plan_check(plan)
    assert rel(ro.cpu().numpy(), oracle.rss(y32, lines, ny, centred=True)) <= OP_TOL


@pytest.mark.parametrize("shape", [(64, 64, 4, 21, 2), (256, 96, 6, 64, 2), (256, 20, 3, 64, 2), (192, 160, 5, 48, 1)],
                         ids=lambda s: "%dx%d" % s[:2])
def test_centred_cg_every_variant_both_modes(shape):
    ny, nx, C, L, F = shape
    x, S, lines, _ = _problem(shape, 9000 + sum(shape))
    S32 = _as32(S)
    y = oracle.forward(_as32(x), S32, lines, centred=True)
    K = 8
    xo, io, _, so = oracle.cg(_as32(y), S32, lines, K, centred=True)
    plan = _plan(S, lines)
    for v in range(sense.NORM_VARIANTS):
        try:
            sense.sense_plan_set_variant(plan, v)
        except sense.SenseError:
            continue
        for mode in (sense.CG_MODE_GRAPH, sense.CG_MODE_PERSISTENT):
            sense.sense_plan_set_cg_mode(plan, mode)
            xg = torch.empty((F, ny, nx), dtype=torch.complex64, device=DEV)
            it = torch.zeros(F, dtype=torch.int32, device=DEV)
            oc = torch.zeros(F, dtype=torch.int32, device=DEV)
            sense.sense_cg_solve(plan, c64(y), c64(S), i32(lines), K, 0.0, xg, it, None, oc)
            sense.sense_plan_check(plan)
            assert rel(xg.cpu().numpy(), xo) <= CG_TOL, (v, mode)
            np.testing.assert_array_equal(it.cpu().numpy(), io)
            np.testing.assert_array_equal(oc.cpu().numpy(), so)


def test_centred_bf16_storage():
    shape = (128, 128, 4, 40, 2)
    ny, nx, C, L, F = shape
    x, S, lines, y = _problem(shape, 9500)
    yq, Sq = oracle.quantize_c64_bf16(y), oracle.quantize_c64_bf16(S)
    plan = _plan(S, lines, sense.STORE_BF16)
    xo = torch.empty((F, ny, nx), dtype=torch.complex64, device=DEV)
    sense.sense_adjoint(plan, bf16_pairs_from_oracle(y), bf16_pairs_from_oracle(S), i32(lines), xo)
    sense.sense_plan_check(plan)
    assert rel(xo.cpu().numpy(), oracle.adjoint(yq, Sq, lines, centred=True)) <= OP_TOL
    xg = torch.empty((F, ny, nx), dtype=torch.complex64, device=DEV)
    sense.sense_cg_solve(plan, bf16_pairs_from_oracle(y), bf16_pairs_from_oracle(S), i32(lines), 6, 0.0, xg)
    sense.sense_plan_check(plan)
    assert rel(xg.cpu().numpy(), oracle.cg(yq, Sq, lines, 6, centred=True)[0]) <= CG_TOL


def test_centred_noalloc_adjoint():
    shape = (96, 64, 3, 30, 2)
    ny, nx, C, L, F = shape
    x, S, lines, y = _problem(shape, 9600)
    xo = torch.empty((F, ny, nx), dtype=torch.complex64, device=DEV)
    sh = dict(ny=ny, nx=nx, coils=C, frames=F, lines=L, centred=1)
    sense.sense_adjoint_noalloc(sh, c64(y), c64(S), i32(lines), xo)
    torch.cuda.synchronize()
    assert rel(xo.cpu().numpy(), oracle.adjoint(_as32(y), _as32(S), lines, centred=True)) <= OP_TOL


def test_centred_batch_and_queue():
    specs = [((64, 64, 4, 21, 2), True), ((64, 64, 3, 16, 1), False), ((128, 96, 5, 40, 2), True)]
    inst = []
    for k, (shape, cen) in enumerate(specs):
        ny, nx, C, L, F = shape
        rng = synth.rng_for(9700 + k)
        S = synth.sensitivities(C, ny, nx)
        lines = synth.mask_lines(ny, L, min(4, L), F, rng)
        if cen:
            lines = synth.centred_lines(lines, ny)
        x = synth.random_complex((F, ny, nx), rng)
        y = oracle.forward(_as32(x), _as32(S), lines, centred=cen)
        inst.append((shape, cen, S, lines, y))
    K = 7
    shapes = [dict(ny=s[0], nx=s[1], coils=s[2], frames=s[4], lines=s[3], centred=int(c)) for s, c, _, _, _ in inst]
    batch = sense.Batch(shapes)
    items = []
    for shape, cen, S, lines, y in inst:
        ny, nx, C, L, F = shape
        items.append(dict(y=c64(y), S=c64(S), lines=i32(lines),
                          x_out=torch.empty((F, ny, nx), dtype=torch.complex64, device=DEV)))
    sense.sense_batch_cg_solve(batch, items, K)
    sense.sense_batch_check(batch)
    torch.cuda.synchronize()
    q = sense.Queue(device=0)
    ids = [q.submit(sh, np.ascontiguousarray(y, np.complex64), np.ascontiguousarray(S, np.complex64),
                    np.ascontiguousarray(lines, np.int32), max_iter=K)
           for sh, (_, _, S, lines, y) in zip(shapes, inst)]
    for k, (shape, cen, S, lines, y) in enumerate(inst):
        ny, nx, C, L, F = shape
        xo = oracle.cg(_as32(y), _as32(S), lines, K, centred=cen)[0]
        assert rel(items[k]["x_out"].cpu().numpy(), xo) <= CG_TOL, k
        xq = np.empty((F, ny, nx), np.complex64)
        q.wait(ids[k], xq)
        assert rel(xq, xo) <= CG_TOL, k
    q.close()
    batch.close()
