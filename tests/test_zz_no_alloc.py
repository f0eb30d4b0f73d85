"""The allocation-free adjoint, sense_adjoint_noalloc, against the plan-based
sense_adjoint (GPU).

Callers that cannot allocate device memory -- plugins whose host owns all
device memory through its own pool, processes with a device memory budget
fixed up front, loops that must stay out of the CUDA allocator -- use the
allocation-free entry point, whose intermediate lives in a fixed file-scope
device array of the library.  This file is named so pytest collects it last;
it passes run alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1807_11830_gb300 import sense, synth
from tests.gpu_util import OP_TOL, c64, ensure_built, i32, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _inputs(seed, ny, nx, C, L, F):
    rng = synth.rng_for(seed)
    S = synth.sensitivities(C, ny, nx)
    lines = synth.mask_lines(ny, L, min(8, L), F, rng)
    y = synth.random_complex((F, C, L, nx), rng)
    return c64(y), c64(S), i32(lines)


def _noalloc_via_c_abi(shape, y, S, lines, x):
    """Call the entry point through the C ABI directly (ctypes, no binding)."""
    lib = sense.load_library()
    sh = sense._Shape(shape["ny"], shape["nx"], shape["coils"], shape["frames"], shape["lines"], 0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.sense_adjoint_noalloc(ctypes.byref(sh), ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(S.data_ptr()),
                                   ctypes.c_void_p(lines.data_ptr()), ctypes.c_void_p(x.data_ptr()), stream)
    return rc


def test_noalloc_adjoint_matches_plan_adjoint_twice():
    ny, nx, C, L, F = 256, 256, 12, 64, 2
    shape = dict(ny=ny, nx=nx, coils=C, frames=F, lines=L)
    plan = sense.Plan(ny, nx, C, F, L)
    for call, seed in enumerate((31, 32)):  # two calls in a row, different data
        y, S, lines = _inputs(seed, ny, nx, C, L, F)
        ref = torch.empty((F, ny, nx), dtype=torch.complex64, device="cuda:0")
        sense.sense_adjoint(plan, y, S, lines, ref)
        got = torch.full((F, ny, nx), float("nan"), dtype=torch.complex64, device="cuda:0")
        assert _noalloc_via_c_abi(shape, y, S, lines, got) == sense.SENSE_OK, call
        torch.cuda.synchronize()
        a = got.cpu().numpy()
        b = ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert rel(a, b) <= OP_TOL, call


def _noalloc_shape(ny, nx, C, L, F, storage):
    return dict(ny=ny, nx=nx, coils=C, frames=F, lines=L, storage=storage)


def _call(shape, y, S, lines, x):
    lib = sense.load_library()
    sh = sense._Shape(shape["ny"], shape["nx"], shape["coils"], shape["frames"], shape["lines"],
                      shape.get("storage", 0))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.sense_adjoint_noalloc(ctypes.byref(sh), ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(S.data_ptr()),
                                     ctypes.c_void_p(lines.data_ptr()), ctypes.c_void_p(x.data_ptr()), stream)


@pytest.mark.parametrize("storage", [sense.STORE_C64, sense.STORE_BF16], ids=["c64", "bf16"])
def test_noalloc_at_its_limit_allocates_nothing(storage):
    """frames * coils * lines * nx exactly at the 2^21 limit (2 x 32 x 128 x
    256), in both storages, against the plan-based adjoint; after a first call
    (which does the one-time set-up and loads the kernels), further calls leave
    the device's free memory and the torch allocator's reservation unchanged."""
    ny, nx, C, L, F = 256, 256, 32, 128, 2
    assert F * C * L * nx == 1 << 21
    shape = _noalloc_shape(ny, nx, C, L, F, storage)
    rng = synth.rng_for(77 + storage)
    S_np = synth.sensitivities(C, ny, nx)
    lines = i32(synth.mask_lines(ny, L, 8, F, rng))
    y_np = synth.random_complex((F, C, L, nx), rng)
    if storage == sense.STORE_C64:
        y, S = c64(y_np), c64(S_np)
    else:
        y, S = sense.to_bf16_pairs(c64(y_np)), sense.to_bf16_pairs(c64(S_np))
    plan = sense.Plan(ny, nx, C, F, L, storage)
    ref = torch.empty((F, ny, nx), dtype=torch.complex64, device="cuda:0")
    sense.sense_adjoint(plan, y, S, lines, ref)
    outs = [torch.full((F, ny, nx), float("nan"), dtype=torch.complex64, device="cuda:0") for _ in range(3)]
    assert _call(shape, y, S, lines, outs[0]) == sense.SENSE_OK
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    for x in outs[1:]:
        assert _call(shape, y, S, lines, x) == sense.SENSE_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0
    b = ref.cpu().numpy()
    for x in outs:
        a = x.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert rel(a, b) <= OP_TOL
