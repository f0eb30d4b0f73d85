"""GPU parity: the CUDA path against the FP64 oracle, element by element.

Tolerances (relative L2 over the whole output): 1e-5 per operator
application in FP32 arithmetic, 1e-4 on the CG image after a fixed number of
iterations.  Shapes span several column tiles, ragged tails (nx smaller than
or not a multiple of the tile width), one line, all lines, non-square
images and every compiled transform length.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1807_11830_gb300 import sense, synth
from tests.gpu_util import (CG_TOL, OP_TOL, ensure_built, gpu_adjoint, gpu_cg, gpu_forward, gpu_normal, gpu_rss,
                            i32, c64, make_plan, rel)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


# (ny, nx, coils, lines, frames)
OP_SHAPES = [
    (8, 8, 2, 3, 2),
    (12, 20, 3, 5, 1),
    (16, 12, 2, 16, 2),
    (20, 16, 3, 1, 1),
    (32, 96, 3, 11, 2),
    (64, 64, 4, 21, 1),
    (96, 160, 2, 30, 1),
    (128, 192, 3, 40, 2),
    (160, 160, 8, 160, 1),
    (192, 128, 5, 48, 2),
    (256, 256, 12, 64, 2),
    (320, 320, 4, 107, 1),
    (384, 384, 3, 64, 1),
    (256, 320, 3, 50, 1),
    (384, 8, 2, 96, 1),
    (24, 40, 2, 9, 2),
    (48, 80, 3, 17, 1),
    (120, 144, 4, 41, 1),
    (144, 120, 3, 48, 2),
    (240, 288, 2, 80, 1),
    (288, 240, 3, 96, 1),
]


def _problem(shape, seed):
    ny, nx, C, L, F = shape
    rng = synth.rng_for(seed)
    S = synth.sensitivities(C, ny, nx)
    lines = synth.mask_lines(ny, L, min(4, L), F, rng)
    x = synth.random_complex((F, ny, nx), rng)
    y = synth.random_complex((F, C, L, nx), rng)
    return x, S, lines, y


@pytest.mark.parametrize("shape", OP_SHAPES, ids=lambda s: "%dx%d_c%d_l%d_f%d" % s)
def test_forward(shape):
    x, S, lines, _ = _problem(shape, 1000 + sum(shape))
    S32 = S.astype(np.complex64).astype(np.complex128)
    x32 = x.astype(np.complex64).astype(np.complex128)
    assert rel(gpu_forward(x, S, lines), oracle.forward(x32, S32, lines)) <= OP_TOL


@pytest.mark.parametrize("shape", OP_SHAPES, ids=lambda s: "%dx%d_c%d_l%d_f%d" % s)
def test_adjoint(shape):
    _, S, lines, y = _problem(shape, 2000 + sum(shape))
    S32 = S.astype(np.complex64).astype(np.complex128)
    y32 = y.astype(np.complex64).astype(np.complex128)
    assert rel(gpu_adjoint(y, S, lines), oracle.adjoint(y32, S32, lines)) <= OP_TOL


@pytest.mark.parametrize("shape", OP_SHAPES, ids=lambda s: "%dx%d_c%d_l%d_f%d" % s)
def test_normal(shape):
    x, S, lines, _ = _problem(shape, 3000 + sum(shape))
    S32 = S.astype(np.complex64).astype(np.complex128)
    x32 = x.astype(np.complex64).astype(np.complex128)
    assert rel(gpu_normal(x, S, lines), oracle.normal(x32, S32, lines)) <= OP_TOL


def _as32(a):
    return a.astype(np.complex64).astype(np.complex128)


def test_eq1_fully_sampled_coil_combine():
    """Eq. 1 of the paper: with every line sampled the adjoint is
    M = sum_i S_i^* F^-1(Y_i); with sum|S|^2 = 1 and Y = E x it returns x."""
    p = synth.single_slice_64()
    n = 64
    lines = synth.full_lines(n, 1)
    y = oracle.forward(p.x_true, p.S, lines)
    m = gpu_adjoint(y, p.S, lines)
    assert rel(m, oracle.adjoint(_as32(y), _as32(p.S), lines)) <= OP_TOL
    assert rel(m, p.x_true) <= 1e-5


def test_cg_single_slice_64():
    p = synth.single_slice_64()
    y = oracle.forward(p.x_true, p.S, p.lines) + p.noise
    xo, io, ro, so = oracle.cg(_as32(y), _as32(p.S), p.lines, p.iters)
    xg, ig, rg, sg = gpu_cg(y, p.S, p.lines, p.iters)
    assert rel(xg, xo) <= CG_TOL
    np.testing.assert_array_equal(ig, io)
    np.testing.assert_array_equal(sg, so)
    np.testing.assert_allclose(rg, ro, rtol=1e-3)


def test_cg_cine_two_frames():
    p = synth.cine_256(frames=20)
    sel = [0, 13]
    x_true = p.x_true[sel]
    lines = p.lines[sel]
    y = oracle.forward(x_true, p.S, lines) + p.noise[sel]
    xo, io, ro, so = oracle.cg(_as32(y), _as32(p.S), lines, p.iters)
    xg, ig, rg, sg = gpu_cg(y, p.S, lines, p.iters)
    assert rel(xg, xo) <= CG_TOL
    np.testing.assert_array_equal(ig, io)
    np.testing.assert_array_equal(sg, so)


def test_cg_stops_at_tolerance():
    p = synth.single_slice_64()
    y = oracle.forward(p.x_true, p.S, p.lines) + p.noise
    tol = 3e-3
    xo, io, ro, so = oracle.cg(_as32(y), _as32(p.S), p.lines, 100, tol)
    xg, ig, rg, sg = gpu_cg(y, p.S, p.lines, 100, tol)
    assert so[0] == sg[0] == sense.CG_CONVERGED
    assert rg[0] <= tol and ro[0] <= tol
    assert abs(int(ig[0]) - int(io[0])) <= 1
    if ig[0] == io[0]:
        assert rel(xg, xo) <= CG_TOL


def test_cg_one_step_exact_recovery():
    """Full sampling and sum|S|^2 = 1 make E^H E = I: one CG step returns x."""
    rng = synth.rng_for(5)
    n, C = 64, 4
    S = synth.sensitivities(C, n, n)
    lines = synth.full_lines(n, 2)
    x = synth.phantom(n, n, 10, rng, frames=2)
    y = oracle.forward(x, S, lines)
    x1, it, rr, oc = gpu_cg(y, S, lines, 1)
    assert rel(x1, x) <= 1e-5 and list(it) == [1, 1]
    xs, it, rr, oc = gpu_cg(y, S, lines, 10, tol=1e-4)
    assert list(it) == [1, 1] and list(oc) == [sense.CG_CONVERGED] * 2 and np.all(rr <= 1e-4)
    assert rel(xs, x) <= 1e-5


def test_cg_zero_frame_and_independence():
    p = synth.cine_256(frames=3)
    y = oracle.forward(p.x_true, p.S, p.lines) + p.noise
    y[1] = 0.0
    xg, ig, rg, sg = gpu_cg(y, p.S, p.lines, 6)
    assert ig[1] == 0 and sg[1] == sense.CG_CONVERGED and rg[1] == 0.0
    assert np.all(xg[1] == 0)
    # frame 2 alone gives the same bits as frame 2 inside the batch
    xa, ia, ra, sa = gpu_cg(y[2:3], p.S, p.lines[2:3], 6)
    np.testing.assert_array_equal(xa[0], xg[2])
    assert ia[0] == ig[2] == 6 and sa[0] == sense.CG_MAXITER


def test_cg_reuses_captured_graph():
    p = synth.single_slice_64()
    y = oracle.forward(p.x_true, p.S, p.lines) + p.noise
    plan = make_plan(p.S, p.lines)
    sense.sense_plan_set_cg_mode(plan, sense.CG_MODE_GRAPH)
    a = gpu_cg(y, p.S, p.lines, 10, plan=plan)
    b = gpu_cg(y, p.S, p.lines, 10, plan=plan)
    np.testing.assert_array_equal(a[0], b[0])


def test_bad_lines_are_flagged():
    x, S, lines, y = _problem((32, 32, 2, 8, 1), 7)
    plan = make_plan(S, lines)
    bad = lines.copy()
    bad[0, 3] = 40  # outside [0, ny)
    out = torch.empty((1, 32, 32), dtype=torch.complex64, device="cuda:0")
    sense.sense_normal(plan, c64(x), c64(S), i32(bad), out)
    with pytest.raises(sense.SenseError) as ei:
        sense.sense_plan_check(plan)
    assert ei.value.status == 9
    unsorted = lines.copy()
    unsorted[0, [2, 3]] = unsorted[0, [3, 2]]
    sense.sense_adjoint(plan, c64(y), c64(S), i32(unsorted), out)
    with pytest.raises(sense.SenseError):
        sense.sense_plan_check(plan)
    sense.sense_plan_check(plan)  # flags were cleared


def test_argument_errors():
    x, S, lines, y = _problem((32, 32, 2, 8, 1), 8)
    plan = make_plan(S, lines)
    xt = c64(x)
    with pytest.raises(sense.SenseError) as ei:
        sense.sense_normal(plan, xt, c64(S), i32(lines), xt)  # out aliases x
    assert ei.value.status == 1
    with pytest.raises(sense.SenseError) as ei:
        sense.Plan(100, 100, 2, 1, 10)
    assert ei.value.status == 2


@pytest.mark.parametrize("shape", [(160, 160, 8, 160, 2), (64, 96, 3, 21, 2)])
def test_rss(shape):
    _, S, lines, y = _problem(shape, 4000 + sum(shape))
    ny = shape[0]
    assert rel(gpu_rss(y, lines, ny), oracle.rss(_as32(y), lines, ny)) <= OP_TOL


def test_paper_workload_full_size():
    """The paper's timed reconstruction at its full shape (16 frames of
    160x160, 8 coils, fully sampled), as the bench runs it: the FFT + RSS
    image and the Eq. 1 combine, every output element against the oracle."""
    p = synth.paper_160()
    S32 = _as32(p.S)
    y = oracle.forward(p.x_true.astype(np.complex64), S32, p.lines) + p.noise
    assert y.shape == (16, 8, 160, 160)
    assert rel(gpu_rss(y, p.lines, 160), oracle.rss(_as32(y), p.lines, 160)) <= OP_TOL
    assert rel(gpu_adjoint(y, p.S, p.lines), oracle.adjoint(_as32(y), S32, p.lines)) <= OP_TOL


VARIANT_SHAPES = [(128, 128, 5, 40, 2), (192, 192, 6, 48, 1), (256, 256, 12, 64, 2), (320, 320, 6, 107, 1),
                  (384, 384, 4, 96, 1), (256, 96, 3, 64, 1), (256, 20, 2, 64, 2)]


@pytest.mark.parametrize("shape", VARIANT_SHAPES, ids=lambda s: "%dx%d_c%d" % s[:3])
def test_normal_every_variant(shape):
    ny, nx, C, L, F = shape
    x, S, lines, _ = _problem(shape, 5000 + sum(shape))
    expect = oracle.normal(_as32(x), _as32(S), lines)
    plan = make_plan(S, lines)
    seen = 0
    for v in range(sense.NORM_VARIANTS):
        try:
            sense.sense_plan_set_variant(plan, v)
        except sense.SenseError:
            continue
        seen += 1
        out = torch.empty((F, ny, nx), dtype=torch.complex64, device="cuda:0")
        sense.sense_normal(plan, c64(x), c64(S), i32(lines), out)
        sense.sense_plan_check(plan)
        assert rel(out.cpu().numpy(), expect) <= OP_TOL, v
    assert seen >= 1


def test_cg_every_variant_and_autotune():
    p = synth.cine_256(frames=3)
    y = oracle.forward(p.x_true, p.S, p.lines) + p.noise
    xo, io, _, _ = oracle.cg(_as32(y), _as32(p.S), p.lines, 8)
    plan = make_plan(p.S, p.lines)
    for v in range(sense.NORM_VARIANTS):
        try:
            sense.sense_plan_set_variant(plan, v)
        except sense.SenseError:
            continue
        for mode in (sense.CG_MODE_GRAPH, sense.CG_MODE_PERSISTENT):
            sense.sense_plan_set_cg_mode(plan, mode)
            xg, ig, _, _ = gpu_cg(y, p.S, p.lines, 8, plan=plan)
            assert rel(xg, xo) <= CG_TOL, (v, mode)
            np.testing.assert_array_equal(ig, io)
    # persistent mode (the default) times short CG solves on scratch buffers
    chosen, times = sense.sense_plan_autotune(plan, c64(p.S), i32(p.lines))
    assert chosen in times and len(times) >= 2
    assert sense.sense_plan_variant(plan) == chosen
    print("autotune persistent 256^2 C12 F3:", chosen, times)
    xg, ig, _, _ = gpu_cg(y, p.S, p.lines, 8, plan=plan)  # the plan's own state is intact
    assert rel(xg, xo) <= CG_TOL
    # the graph mode is timed (and cached) separately, per launch
    sense.sense_plan_set_cg_mode(plan, sense.CG_MODE_GRAPH)
    chosen_g, times_g = sense.sense_plan_autotune(plan, c64(p.S), i32(p.lines))
    assert chosen_g in times_g and set(times_g) == set(times)
    assert max(times_g.values()) < min(times.values())  # one launch vs ten iterations
    print("autotune graph 256^2 C12 F3:", chosen_g, times_g)
    xg, ig, _, _ = gpu_cg(y, p.S, p.lines, 8, plan=plan)
    assert rel(xg, xo) <= CG_TOL


@pytest.mark.parametrize("shape", [(256, 20, 3, 64, 2), (128, 12, 4, 40, 3), (192, 20, 5, 48, 2),
                                   (320, 20, 3, 107, 2)],
                         ids=lambda s: "%dx%d" % s[:2])
def test_cg_every_variant_ragged_tiles(shape):
    """Image widths that leave the last column tile (and, for lane-major
    variants, whole warps) partly empty: every variant, both CG modes."""
    ny, nx, C, L, F = shape
    x, S, lines, _ = _problem(shape, 7000 + sum(shape))
    S32 = _as32(S)
    y = oracle.forward(_as32(x), S32, lines)
    xo, io, _, _ = oracle.cg(_as32(y), S32, lines, 6)
    plan = make_plan(S, lines)
    for v in range(sense.NORM_VARIANTS):
        try:
            sense.sense_plan_set_variant(plan, v)
        except sense.SenseError:
            continue
        for mode in (sense.CG_MODE_GRAPH, sense.CG_MODE_PERSISTENT):
            sense.sense_plan_set_cg_mode(plan, mode)
            xg, ig, _, _ = gpu_cg(y, S, lines, 6, plan=plan)
            assert rel(xg, xo) <= CG_TOL, (v, mode)


@pytest.mark.parametrize("which", ["slice64", "cine256", "slices320", "mix192"])
def test_cg_both_modes_match_oracle(which):
    """The persistent single-launch CG and the per-phase graph CG both match
    the oracle; iteration counts and outcomes agree."""
    if which == "slice64":
        p = synth.single_slice_64()
        sel, K = [0], 10
    elif which == "cine256":
        p = synth.cine_256(frames=4)
        sel, K = [0, 1, 2, 3], 12
    elif which == "slices320":
        p = synth.slices_320(frames=2)
        sel, K = [0, 1], 6
    else:
        p = synth.mix_instance(dict(n=192, coils=9, frames=3, accel=3, lines=64, centre=12), 77)
        sel, K = [0, 1, 2], 15
    y = oracle.forward(p.x_true[sel], p.S, p.lines[sel]) + p.noise[sel]
    lines = p.lines[sel]
    xo, io, _, so = oracle.cg(_as32(y), _as32(p.S), lines, K)
    for mode in (sense.CG_MODE_PERSISTENT, sense.CG_MODE_GRAPH):
        plan = make_plan(p.S, lines)
        sense.sense_plan_set_cg_mode(plan, mode)
        xg, ig, _, sg = gpu_cg(y, p.S, lines, K, plan=plan)
        assert rel(xg, xo) <= CG_TOL, mode
        np.testing.assert_array_equal(ig, io)
        np.testing.assert_array_equal(sg, so)


def test_cg_persistent_tolerance_stop():
    p = synth.cine_256(frames=3)
    y = oracle.forward(p.x_true, p.S, p.lines) + p.noise
    tol = 2e-3
    xo, io, ro, so = oracle.cg(_as32(y), _as32(p.S), p.lines, 60, tol)
    plan = make_plan(p.S, p.lines)
    sense.sense_plan_set_cg_mode(plan, sense.CG_MODE_PERSISTENT)
    xg, ig, rg, sg = gpu_cg(y, p.S, p.lines, 60, tol=tol, plan=plan)
    assert np.all(sg == sense.CG_CONVERGED) and np.all(rg <= tol)
    assert np.all(np.abs(ig.astype(int) - io.astype(int)) <= 1)


def test_bounded_wait_gives_up_and_device_stays_usable():
    assert sense.sense_selftest_wait(0, 2000) == 5  # SENSE_ETIMEOUT
    p = synth.single_slice_64()
    y = oracle.forward(p.x_true, p.S, p.lines) + p.noise
    xg, ig, _, _ = gpu_cg(y, p.S, p.lines, 3)
    assert list(ig) == [3]


@pytest.mark.parametrize("n", sense.SIZES)
def test_cg_persistent_every_length(n):
    """Persistent CG (maps staged into shared memory by TMA) at every
    compiled length, including tiles wider than the image (nx < 16)."""
    rng = synth.rng_for(7000 + n)
    C, F = 3, 2
    L = max(1, n // 3)
    S = synth.sensitivities(C, n, n)
    lines = synth.mask_lines(n, L, min(4, L), F, rng)
    x = synth.random_complex((F, n, n), rng)
    y = oracle.forward(x, S, lines)
    K = 6
    xo, io, _, so = oracle.cg(_as32(y), _as32(S), lines, K)
    plan = make_plan(S, lines)
    sense.sense_plan_set_cg_mode(plan, sense.CG_MODE_PERSISTENT)
    xg, ig, _, sg = gpu_cg(y, S, lines, K, plan=plan)
    assert rel(xg, xo) <= CG_TOL
    np.testing.assert_array_equal(ig, io)


@pytest.mark.parametrize("storage", [sense.STORE_C64, sense.STORE_BF16])
def test_cg_solve_host_equals_device_call(storage):
    """sense_cg_solve_host (host buffers in and out) gives the device call's
    bits: the same kernels on the same data; two calls in a row reuse the
    plan's device copies."""
    from tests.gpu_util import storage_tensor

    ny, nx, C, L, F = 192, 128, 5, 48, 3
    x, S, lines, y = _problem((ny, nx, C, L, F), seed=4242 + storage)
    plan = make_plan(S, lines, storage)
    xd, itd, rrd, ocd = gpu_cg(y, S, lines, 12, plan=plan, storage=storage)
    y_t = storage_tensor(y, storage).cpu().pin_memory()
    S_t = storage_tensor(S, storage).cpu().pin_memory()
    l_t = torch.from_numpy(np.ascontiguousarray(lines, np.int32)).pin_memory()
    for _ in range(2):
        xh = torch.empty((F, ny, nx), dtype=torch.complex64).pin_memory()
        ith = torch.zeros(F, dtype=torch.int32)
        rrh = torch.zeros(F, dtype=torch.float64)
        och = torch.zeros(F, dtype=torch.int32)
        sense.sense_cg_solve_host(plan, y_t, S_t, l_t, 12, 0.0, xh, ith, rrh, och)
        np.testing.assert_array_equal(xh.numpy().astype(np.complex128), xd)
        np.testing.assert_array_equal(ith.numpy(), itd)
        np.testing.assert_array_equal(rrh.numpy(), rrd)
        np.testing.assert_array_equal(och.numpy(), ocd)
