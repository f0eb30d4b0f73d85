"""Guard bands around every output buffer (GPU).

No device sanitizer runs on this hardware, so out-of-range writes are
caught this way.  Each output is placed inside a larger buffer whose bands
before and after it hold a canary bit pattern.  After each call:
  * every guard word is unchanged, so nothing was written outside the output;
  * no interior word still holds the canary, so every output element was written;
  * every input (y, S, lines, x) is bit for bit unchanged.
Shapes are non-square with ragged column and row tiles; uncentred, centred
and BF16 storage are all covered.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1807_11830_gb300 import sense, synth
from tests.gpu_util import DEV, bf16_pairs_from_oracle, c64, ensure_built, i32

pytestmark = pytest.mark.gpu

CANARY = 0x7FC0DEAD  # a quiet NaN with a recognisable payload
GUARD_BYTES = 2048


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


class Guarded:
    """A tensor view of `shape`/`dtype` inside a canary-filled int32 buffer."""

    def __init__(self, shape, dtype):
        elem = torch.empty((), dtype=dtype).element_size()
        self.nbytes = int(np.prod(shape)) * elem
        body_words = (self.nbytes + 3) // 4
        g = GUARD_BYTES // 4
        self.words = torch.full((g + body_words + g,), CANARY, dtype=torch.int32, device=DEV)
        self.g = g
        self.body_words = body_words
        raw = self.words[g:g + body_words].view(torch.uint8)[: self.nbytes]
        self.view = raw.view(dtype).view(shape)

    def check(self, what, fully_written=True):
        w = self.words.cpu().numpy()
        g, b = self.g, self.body_words
        assert np.all(w[:g] == CANARY), "%s: write before the output" % what
        assert np.all(w[g + b:] == CANARY), "%s: write after the output" % what
        if fully_written:
            assert not np.any(w[g:g + b] == CANARY), "%s: output element left unwritten" % what


def _bits(t):
    return t.contiguous().view(torch.uint8).cpu().numpy().copy()


SHAPES = [  # ny, nx, coils, frames, lines, centred, storage
    (48, 80, 3, 2, 17, 0, sense.STORE_C64),
    (160, 120, 5, 3, 41, 1, sense.STORE_C64),
    (256, 24, 2, 1, 64, 0, sense.STORE_C64),
    (96, 40, 4, 2, 30, 0, sense.STORE_BF16),
    (20, 384, 3, 2, 9, 1, sense.STORE_C64),
]


def _inputs(ny, nx, C, F, L, storage, seed):
    rng = synth.rng_for(seed)
    S = synth.sensitivities(C, ny, nx)
    lines = synth.mask_lines(ny, L, min(4, L), F, rng)
    x = synth.random_complex((F, ny, nx), rng)
    y = synth.random_complex((F, C, L, nx), rng)
    if storage == sense.STORE_BF16:
        return bf16_pairs_from_oracle(S), i32(lines), c64(x), bf16_pairs_from_oracle(y)
    return c64(S), i32(lines), c64(x), c64(y)


@pytest.mark.parametrize("spec", SHAPES, ids=lambda s: "%dx%d_c%d_f%d_l%d_%s_%s" % (
    s[0], s[1], s[2], s[3], s[4], "centred" if s[5] else "dc0", "bf16" if s[6] else "c64"))
def test_outputs_stay_in_bounds(spec):
    ny, nx, C, F, L, centred, storage = spec
    S, lines, x, y = _inputs(ny, nx, C, F, L, storage, 7000 + ny + nx)
    before = {k: _bits(v) for k, v in dict(S=S, lines=lines, x=x, y=y).items()}
    plan = sense.Plan(ny, nx, C, F, L, storage, centred=bool(centred))
    ydt = torch.complex64 if storage == sense.STORE_C64 else torch.bfloat16
    yshape = (F, C, L, nx) if storage == sense.STORE_C64 else (F, C, L, nx, 2)

    out = Guarded(yshape, ydt)
    sense.sense_forward(plan, x, S, lines, out.view)
    sense.sense_plan_check(plan)
    out.check("forward")

    out = Guarded((F, ny, nx), torch.complex64)
    sense.sense_adjoint(plan, y, S, lines, out.view)
    sense.sense_plan_check(plan)
    out.check("adjoint")

    out = Guarded((F, ny, nx), torch.complex64)
    sense.sense_normal(plan, x, S, lines, out.view)
    sense.sense_plan_check(plan)
    out.check("normal")

    out = Guarded((F, ny, nx), torch.float32)
    sense.sense_rss(plan, y, lines, out.view)
    sense.sense_plan_check(plan)
    out.check("rss")

    shape = dict(ny=ny, nx=nx, coils=C, frames=F, lines=L, storage=storage, centred=centred)
    out = Guarded((F, ny, nx), torch.complex64)
    sense.sense_adjoint_noalloc(shape, y, S, lines, out.view)
    torch.cuda.synchronize()
    out.check("adjoint_noalloc")

    for mode in (sense.CG_MODE_GRAPH, sense.CG_MODE_PERSISTENT):
        sense.sense_plan_set_cg_mode(plan, mode)
        xo = Guarded((F, ny, nx), torch.complex64)
        it = Guarded((F,), torch.int32)
        rr = Guarded((F,), torch.float64)
        oc = Guarded((F,), torch.int32)
        sense.sense_cg_solve(plan, y, S, lines, 5, 0.0, xo.view, it.view, rr.view, oc.view)
        sense.sense_plan_check(plan)
        for g, name in ((xo, "x"), (it, "iters"), (rr, "resid"), (oc, "outcome")):
            g.check("cg mode %d %s" % (mode, name))

    after = {k: _bits(v) for k, v in dict(S=S, lines=lines, x=x, y=y).items()}
    for k in before:
        np.testing.assert_array_equal(before[k], after[k], err_msg="input %s modified" % k)


def test_batch_outputs_stay_in_bounds():
    specs = [(64, 64, 3, 2, 22), (128, 128, 4, 1, 43), (64, 64, 2, 3, 16)]
    items, guards, keep = [], [], []
    shapes = []
    for k, (ny, nx, C, F, L) in enumerate(specs):
        S, lines, _, _ = _inputs(ny, nx, C, F, L, sense.STORE_C64, 7100 + k)
        rng = synth.rng_for(7200 + k)
        xt = synth.random_complex((F, ny, nx), rng)
        y = c64(oracle.forward(xt, S.cpu().numpy(), lines.cpu().numpy()))
        g = dict(x_out=Guarded((F, ny, nx), torch.complex64), iters_out=Guarded((F,), torch.int32),
                 rel_resid_out=Guarded((F,), torch.float64), outcome_out=Guarded((F,), torch.int32))
        items.append(dict(y=y, S=S, lines=lines, **{n: v.view for n, v in g.items()}))
        guards.append(g)
        keep.append({n: _bits(t) for n, t in dict(y=y, S=S, lines=lines).items()})
        shapes.append(dict(ny=ny, nx=nx, coils=C, frames=F, lines=L))
    batch = sense.Batch(shapes)
    sense.sense_batch_cg_solve(batch, items, 6)
    sense.sense_batch_check(batch)
    torch.cuda.synchronize()
    for k, g in enumerate(guards):
        for name, gd in g.items():
            gd.check("batch instance %d %s" % (k, name))
        for name in ("y", "S", "lines"):
            np.testing.assert_array_equal(keep[k][name], _bits(items[k][name]))
    batch.close()
