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
