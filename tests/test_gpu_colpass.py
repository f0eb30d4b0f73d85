"""The three ways E, E^H and root-sum-of-squares can run against the FP64
oracle (sense_plan_set_column_pass): 1 (the default), two launches with the
persistent TMA-staged column pass; 2, both passes in one persistent launch
with a frame-staggered schedule (square images of a length with a TMA column
pass); 0, two launches with the per-tile column kernels.

Shapes cover every length with a TMA column pass, ragged column tails (nx not
a multiple of 8), more (frame, tile) items than resident blocks (so blocks
loop and prefetch across items), more than 256 lines (two k-space boxes),
centred k-space, BF16 storage, the CG start (mode 1) through a short CG
solve, and the paper's fully sampled 160x160 reconstruction."""
import numpy as np
import pytest
import torch

import oracle
from paper_1807_11830_gb300 import sense, synth
from tests.gpu_util import (CG_TOL, DEV, OP_TOL, bf16_pairs_to_complex, c64, ensure_built, i32, rel,
                            storage_tensor)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _as32(a):
    return np.asarray(a).astype(np.complex64).astype(np.complex128)


def _problem(ny, nx, C, L, F, seed):
    rng = synth.rng_for(seed)
    S = synth.sensitivities(C, ny, nx)
    lines = synth.mask_lines(ny, L, min(4, L), F, rng)
    x = synth.random_complex((F, ny, nx), rng)
    y = synth.random_complex((F, C, L, nx), rng)
    return x, S, lines, y


def _plan(S, lines, staged, storage=sense.STORE_C64, centred=False):
    C, ny, nx = S.shape
    F, L = lines.shape
    plan = sense.Plan(ny, nx, C, F, L, storage, centred=centred)
    sense.sense_plan_set_column_pass(plan, staged)
    return plan


# (ny, nx, coils, lines, frames)
SHAPES = [
    (64, 64, 4, 21, 40),      # 320 items: blocks loop over several items
    (96, 20, 3, 30, 3),       # ragged: 20 columns = 2 full tiles + 4
    (120, 144, 3, 41, 2),
    (128, 128, 5, 40, 2),
    (144, 120, 3, 48, 2),
    (160, 160, 8, 160, 2),
    (192, 128, 5, 48, 2),
    (240, 96, 2, 80, 1),
    (256, 256, 12, 64, 3),
    (288, 240, 3, 96, 1),
    (320, 320, 6, 300, 1),    # 300 lines: two k-space boxes per coil
    (384, 384, 3, 384, 1),    # every line
    (384, 12, 2, 96, 30),     # 30 frames x 2 tiles, 12 columns
]
IDS = ["%dx%d_c%d_l%d_f%d" % s for s in SHAPES]


@pytest.mark.parametrize("staged", [2, 1, 0])
@pytest.mark.parametrize("shape", SHAPES, ids=IDS)
def test_forward_and_adjoint_both_column_passes(shape, staged):
    x, S, lines, y = _problem(*shape, seed=7000 + sum(shape))
    ny, nx, C, L, F = shape
    plan = _plan(S, lines, staged)
    yo = torch.empty((F, C, L, nx), dtype=torch.complex64, device=DEV)
    xa = torch.empty((F, ny, nx), dtype=torch.complex64, device=DEV)
    sense.sense_forward(plan, c64(x), c64(S), i32(lines), yo)
    sense.sense_adjoint(plan, c64(y), c64(S), i32(lines), xa)
    sense.sense_plan_check(plan)
    assert rel(yo.cpu().numpy(), oracle.forward(_as32(x), _as32(S), lines)) <= OP_TOL
    assert rel(xa.cpu().numpy(), oracle.adjoint(_as32(y), _as32(S), lines)) <= OP_TOL


@pytest.mark.parametrize("shape", [(256, 256, 4, 64, 2), (320, 192, 3, 107, 2), (160, 160, 8, 160, 2)],
                         ids=lambda s: "%dx%d" % s[:2])
def test_centred_and_bf16(shape):
    x, S, lines, y = _problem(*shape, seed=7100 + sum(shape))
    ny, nx, C, L, F = shape
    cl = synth.centred_lines(lines, ny)
    plan = _plan(S, cl, 1, centred=True)
    yo = torch.empty((F, C, L, nx), dtype=torch.complex64, device=DEV)
    xa = torch.empty((F, ny, nx), dtype=torch.complex64, device=DEV)
    sense.sense_forward(plan, c64(x), c64(S), i32(cl), yo)
    sense.sense_adjoint(plan, c64(y), c64(S), i32(cl), xa)
    sense.sense_plan_check(plan)
    assert rel(yo.cpu().numpy(), oracle.forward(_as32(x), _as32(S), cl, centred=True)) <= OP_TOL
    assert rel(xa.cpu().numpy(), oracle.adjoint(_as32(y), _as32(S), cl, centred=True)) <= OP_TOL
    q = oracle.quantize_c64_bf16
    bplan = _plan(S, lines, 1, storage=sense.STORE_BF16)
    xb = torch.empty((F, ny, nx), dtype=torch.complex64, device=DEV)
    sense.sense_adjoint(bplan, storage_tensor(y, sense.STORE_BF16), storage_tensor(S, sense.STORE_BF16), i32(lines),
                        xb)
    yb = torch.empty((F, C, L, nx, 2), dtype=torch.bfloat16, device=DEV)
    sense.sense_forward(bplan, c64(x), storage_tensor(S, sense.STORE_BF16), i32(lines), yb)
    sense.sense_plan_check(bplan)
    assert rel(xb.cpu().numpy(), oracle.adjoint(q(y), q(S), lines)) <= OP_TOL
    assert rel(bf16_pairs_to_complex(yb), oracle.forward(_as32(x), q(S), lines)) <= 2.0 ** -8
    # the single-launch form on the same centred and BF16 problems
    fplan = _plan(S, cl, 2, centred=True)
    sense.sense_adjoint(fplan, c64(y), c64(S), i32(cl), xa)
    sense.sense_plan_check(fplan)
    assert rel(xa.cpu().numpy(), oracle.adjoint(_as32(y), _as32(S), cl, centred=True)) <= OP_TOL
    fb = _plan(S, lines, 2, storage=sense.STORE_BF16)
    sense.sense_forward(fb, c64(x), storage_tensor(S, sense.STORE_BF16), i32(lines), yb)
    sense.sense_plan_check(fb)
    assert rel(bf16_pairs_to_complex(yb), oracle.forward(_as32(x), q(S), lines)) <= 2.0 ** -8


@pytest.mark.parametrize("shape", [(160, 160, 8, 160, 16), (256, 192, 4, 64, 3), (384, 384, 2, 300, 1)],
                         ids=lambda s: "%dx%d_l%d" % (s[0], s[1], s[3]))
def test_rss_both_column_passes(shape):
    _, _, lines, y = _problem(*shape, seed=7200 + sum(shape))
    ny, nx, C, L, F = shape
    ref = oracle.rss(_as32(y), lines, ny)
    for staged in (2, 1, 0):
        plan = sense.Plan(ny, nx, C, F, L)
        sense.sense_plan_set_column_pass(plan, staged)
        out = torch.empty((F, ny, nx), dtype=torch.float32, device=DEV)
        sense.sense_rss(plan, c64(y), i32(lines), out)
        sense.sense_plan_check(plan)
        assert rel(out.cpu().numpy(), ref) <= OP_TOL


@pytest.mark.parametrize("shape", [(256, 256, 12, 64, 3), (320, 320, 8, 107, 2), (192, 96, 5, 48, 2)],
                         ids=lambda s: "%dx%d" % s[:2])
def test_cg_start_both_column_passes(shape):
    """The CG start (b = E^H y into r and p, rho0) runs in the column pass:
    a 6-iteration CG from either pass matches the oracle, with the same
    iteration counts."""
    _, S, lines, y = _problem(*shape, seed=7300 + sum(shape))
    ny, nx, C, L, F = shape
    xo, io, _, _ = oracle.cg(_as32(y), _as32(S), lines, 6)
    for staged in (2, 1, 0):
        plan = _plan(S, lines, staged)
        x = torch.empty((F, ny, nx), dtype=torch.complex64, device=DEV)
        it = torch.zeros(F, dtype=torch.int32, device=DEV)
        sense.sense_cg_solve(plan, c64(y), c64(S), i32(lines), 6, 0.0, x, it)
        sense.sense_plan_check(plan)
        assert rel(x.cpu().numpy(), xo) <= CG_TOL
        np.testing.assert_array_equal(it.cpu().numpy(), io)


@pytest.mark.parametrize("shape", [(256, 256, 12, 64, 20), (160, 160, 8, 160, 16), (128, 128, 3, 33, 1)],
                         ids=lambda s: "%dx%d_f%d" % (s[0], s[1], s[4]))
def test_fused_equals_two_launch_results(shape):
    """The single-launch schedule gives the two-launch TMA results to the bit
    for E (no sums differ) and within rounding for E^H, RSS and the CG start,
    with many frames (so tiles of several frames are in flight at once)."""
    x, S, lines, y = _problem(*shape, seed=7400 + sum(shape))
    ny, nx, C, L, F = shape
    res = {}
    for staged in (2, 1):
        plan = _plan(S, lines, staged)
        yo = torch.empty((F, C, L, nx), dtype=torch.complex64, device=DEV)
        xa = torch.empty((F, ny, nx), dtype=torch.complex64, device=DEV)
        ro = torch.empty((F, ny, nx), dtype=torch.float32, device=DEV)
        sense.sense_forward(plan, c64(x), c64(S), i32(lines), yo)
        sense.sense_adjoint(plan, c64(y), c64(S), i32(lines), xa)
        sense.sense_rss(plan, c64(y), i32(lines), ro)
        sense.sense_plan_check(plan)
        res[staged] = (yo.cpu().numpy(), xa.cpu().numpy(), ro.cpu().numpy())
    np.testing.assert_array_equal(res[2][0], res[1][0])
    assert rel(res[2][1], res[1][1]) <= 1e-6
    assert rel(res[2][2], res[1][2]) <= 1e-6
